"""GB300-native grouped-qubit MPS TEBD of the 2D transverse-field Ising model.

The compute path is the CUDA library ``libmpsgb.so`` (C ABI in include/mpsgb.h),
built in-tree by ``paper_2511_23438_gb300.build.build()``; ``paper_2511_23438_gb300.lib``
is a thin ctypes binding with the same names.  Importing the package does not
load the library; ``lib.load()`` does, and fails loudly if it is missing.
"""
__all__ = ["lib", "build", "inputs", "serve"]
