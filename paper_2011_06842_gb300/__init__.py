"""GB300 (sm_103a) implementation of the augmented FEWHA hot path
(Ramlau & Stadler, "An augmented wavelet reconstructor for atmospheric
tomography"): the matrix-free FEWHA normal operator and the (augmented) PCG
time step, as CUDA kernels behind the C ABI in include/fewha.h.

``fewha`` is the Python binding (argument marshalling only); ``build`` compiles
libfewha.so in-tree; ``workload`` holds the paper's FLOP model and the
algorithmic byte counts used for the roofline.
"""
from .fewha import (Fewha, FewhaBatch, FewhaError, FewhaState, McaoFit, autotune_batch, exported_symbols,  # noqa: F401
                    load_library, make_geometry, read_bandwidth)
