"""GB300 (sm_103a) implementation of the augmented FEWHA hot path
(Ramlau & Stadler, "An augmented wavelet reconstructor for atmospheric
tomography"): the matrix-free FEWHA normal operator and the (augmented) PCG
time step, as CUDA kernels behind the C ABI in include/fewha.h.

``fewha`` is the Python binding (argument marshalling only); ``build`` compiles
libfewha.so in-tree; ``workload`` holds the paper's FLOP model and the
algorithmic byte counts used for the roofline.
"""
from .fewha import (Fewha, FewhaError, FewhaState, exported_symbols, load_library,  # noqa: F401
                    make_geometry)
