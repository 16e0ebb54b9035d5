"""GB300-native two-level nonlinear Schwarz solver (arXiv 2410.24138), sm_103a CUDA behind a C ABI.

``paper_2410_24138_gb300.nls`` is the Python binding of the C-ABI library ``libnls.so``
(built in-tree by ``paper_2410_24138_gb300.build``); it is imported lazily so that the
seeded input generators in ``paper_2410_24138_gb300.inputs`` load without a GPU.
"""
