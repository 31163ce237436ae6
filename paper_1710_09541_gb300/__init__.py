"""GB300-native phase-field lattice Boltzmann step (arXiv:1710.09541).

The compute path is the CUDA library ``_lib/liblbm_pf.so`` (sm_103a) behind
the C ABI declared in ``include/lbm_pf.h``; ``lbm`` is its thin ctypes binding.
"""
