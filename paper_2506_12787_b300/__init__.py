"""B300 (sm_103a) implementation of SwiftWRF spectrum synthesis
(arXiv 2506.12787): deformation MLP over 2D Gaussians, projection, tile
binning and an order-free tile rasteriser, behind the C ABI in include/wrf.h.
"""
from ._lib import WrfError, load  # noqa: F401

__version__ = "0.1.0"
