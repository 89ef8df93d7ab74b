"""GB300-native stratified Monte Carlo integration with heuristic tree search
(the method of ZMCintegral, arXiv 1902.07916).

The compute path is libzmc.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/zmc.h); ``zmc`` is its Python binding, ``workloads`` the seeded
synthetic workload definitions, ``build`` the in-tree nvcc build.
"""
from . import build  # noqa: F401


def load():
    """Import the binding (raises ImportError if libzmc.so was not built)."""
    from . import zmc
    return zmc
