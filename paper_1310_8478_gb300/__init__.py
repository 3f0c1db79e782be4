"""GB300 engine for the per-millisecond step of the DPSNN-STDP mini-application
(Paolucci et al., arXiv 1310.8478): CUDA kernels for sm_103a behind the C ABI
of include/snn.h, with a ctypes binding."""
from .snn import (  # noqa: F401
    Network, Batch, SnnError, load, library_path, make_config,
    snn_build_network, snn_build_network_explicit, snn_step, snn_run, snn_free,
    snn_read_raster, snn_read_weights, STDP_OFF, DELIVERY_OFF,
)
from .build import build as build_engine  # noqa: F401
from . import snn  # noqa: F401
