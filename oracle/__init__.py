"""CPU oracle for the Gaussian RBF interpolation solve (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the CUDA library never does.
"""
