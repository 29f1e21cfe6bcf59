"""B300-native mapped Legendre / Fourier spectral transform pair (sm_103a).

The compute path lives in the C-ABI shared library ``libmlx.so`` built from
``csrc/``; ``binding`` marshals arguments to it.  Importing this package does not
load the library (so the seeded input generators in ``workloads`` stay usable on a
machine without a GPU); the first call into ``binding`` does, and fails loudly if
the library is missing.
"""
