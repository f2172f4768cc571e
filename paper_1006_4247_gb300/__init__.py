"""GB300-native parallel tempering for the 3D Heisenberg spin glass.

Hot path (checkerboard heat-bath and overrelaxation sweeps, energy and overlap
reductions, standard / decimation / cooling-heating replica exchange of
Hasenbusch & Schaefer, arXiv:1006.4247) in hand-written CUDA for sm_103a
behind the C ABI of include/pt.h; ``pt`` is its Python binding.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pt", "build"]


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
