"""GB300-native D2Q9 generalized Onsager-regularised lattice Boltzmann (arXiv 2602.21242).

The compute path is the CUDA C-ABI library ``liblbm.so`` (sources in ``csrc/``,
declarations in ``include/lbm.h``); ``capi`` binds it through ctypes and
``lattice`` wraps it for torch tensors, ``slab`` splits one lattice over ranks. Nothing here computes lattice
Boltzmann arithmetic in Python.
"""
__all__ = ["capi", "lattice", "flows", "slab"]
