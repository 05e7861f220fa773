"""GB300-native Greedy Frank-Wolfe graph segmentation (arXiv 2508.09738).

`binding`   -- ctypes binding of the C ABI in include/fw_seg.h (CUDA library)
`build`     -- in-tree nvcc build of the library for sm_103a
`workloads` -- seeded synthetic inputs (graphs, labels); no method arithmetic

Importing the package loads nothing; the CUDA library is loaded on first use.
"""
__all__ = ["binding", "build", "workloads"]
