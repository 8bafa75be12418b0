"""GB300-native hierarchical Q~v / Q~^T w for rigid bodies (arXiv 1708.08427).

The compute path is the CUDA library ``libzq.so`` (C ABI, ``include/zq.h``);
``paper_1708_08427_gb300.zq`` is its ctypes binding.  Importing this package
does not load the library; ``paper_1708_08427_gb300.workloads`` only draws
synthetic inputs.
"""
__all__ = ["workloads", "zq"]
