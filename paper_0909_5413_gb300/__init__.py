"""GB300 Gaussian RBF interpolation: GMRES + restricted additive Schwarz,
cell-list truncated matvec, all in hand-written CUDA behind a C ABI.

``rbf`` is the ctypes binding of ``librbf.so``; ``workloads`` draws seeded
synthetic inputs; ``build`` compiles the library for sm_103a.
"""
