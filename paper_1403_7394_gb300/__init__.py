"""GB300-native Hierarchical Affinity Propagation (arXiv:1403.7394).

The CUDA library (libhap.so, C ABI in include/hap.h) holds the whole hot
path; ``paper_1403_7394_gb300.hap`` is its Python binding and loads the
library on import.  ``workloads`` holds seeded synthetic point sets.
"""
__all__ = ["hap", "workloads", "build"]
