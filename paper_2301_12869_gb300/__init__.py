"""GB300 (sm_103a) D2Q9 pseudopotential lattice Boltzmann step.

The compute path is the ``liblbm`` shared library (hand-written CUDA behind a
C ABI, declared in ``include/lbm.h``); ``paper_2301_12869_gb300.lbm`` is its
thin ctypes binding and ``paper_2301_12869_gb300.inputs`` draws the seeded
synthetic inputs.
"""
