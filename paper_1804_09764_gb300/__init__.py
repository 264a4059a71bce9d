"""GB300 (sm_103a) colour-coding counter for non-induced tree templates.

Method: arXiv 1804.09764, Section 2.1 (Eq. 1, Algorithm 1, Eq. 3), with the
neighbour-list partitioning of Algorithm 4 in its one-GPU form.

Modules:
  graphgen  seeded synthetic graphs and templates (inputs only)
  build     nvcc build of the CUDA library (in-tree, sm_103a)
  cc        ctypes binding of the C ABI (include/cc.h)
"""
__all__ = ["graphgen", "build", "cc"]
