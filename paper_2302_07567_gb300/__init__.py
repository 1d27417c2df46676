"""GB300-native relativistic space-charge FMM (barycentric Lagrange dual tree traversal).

The compute path is the CUDA library built from ``csrc/`` and reached
through the C ABI declared in ``include/fmm.h``; ``fmm`` is its Python
binding.  Importing the package does not load the library, so the input
generators in ``workloads`` stay usable on machines without a GPU; the
first call into ``fmm`` loads it and raises if it is missing.
"""
__all__ = ["workloads", "fmm"]
