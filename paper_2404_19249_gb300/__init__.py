"""GB300 (sm_103a) implementation of the fine-mesh hot path of the nonnested
augmented subspace method for the Kohn-Sham equation (arXiv 2404.19249).

The compute lives in the native library libnas.so (C ABI in include/nas.h);
`paper_2404_19249_gb300.nas` is its ctypes binding.  Build the library with
`python -m paper_2404_19249_gb300.build`.
"""
__all__ = ["nas", "build"]
