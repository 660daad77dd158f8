"""GB300-native parallel cross-validation for Gaussian-process models (arXiv 1912.13132).

The hot path lives in the CUDA library behind include/pcv.h; ``pcv`` is its
Python binding and ``datagen`` the seeded synthetic inputs.
"""
__all__ = ["pcv", "datagen", "build_ext"]
