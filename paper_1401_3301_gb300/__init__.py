"""GB300-native P1 finite element assembly (after Cuvelier, Japhet, Scarella).

``fe`` is the binding of the C ABI (include/fe.h); ``meshgen`` makes seeded
synthetic meshes and coefficient fields. Importing the package does not load
the CUDA library; the first call into ``fe`` does.
"""
from . import meshgen  # noqa: F401
