"""GB300-native domain-wall fermion operator (Shamir and Moebius).

The compute path is the CUDA library libdw_gb300.so (sources in csrc/, C ABI
in include/dw.h); :mod:`.dw` binds it with ctypes, :mod:`.lattice` adds
PyTorch-allocated device fields, :mod:`.inputs` generates the seeded
synthetic gauge and spinor fields, and :mod:`.build` compiles the library.
Importing this package loads nothing; the library is loaded on first use and
its absence is an error.
"""

__all__ = ["build", "dw", "inputs", "lattice"]
