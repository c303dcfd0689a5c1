"""B300-native generalized Laguerre cells, partial-OT Newton solve and fluid step.

The compute path is the CUDA library libpot.so (csrc/, C ABI in include/pot.h);
`pot` is its thin ctypes binding and `scenes` the seeded input generators.
Importing the package loads nothing; the library is opened on first use and
every entry point fails loudly if it is missing.
"""
__all__ = ["pot", "scenes"]
