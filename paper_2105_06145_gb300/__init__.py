"""GB300-native stepping SSSP (rho-Stepping, Delta*-Stepping, Bellman-Ford).

Exact single-source shortest paths by the stepping framework of Dong, Gu, Sun,
Zhang (SPAA'21), run as one persistent CUDA kernel per solve on sm_103a.

Submodules:
  sssp      -- ctypes binding of libsssp.so (the C ABI in include/sssp.h)
  graphgen  -- seeded synthetic CSR graphs (input side only)
  build     -- nvcc build of libsssp.so

The binding is imported lazily (``from paper_2105_06145_gb300 import sssp``)
so that the input generators can be used without the CUDA library.
"""
__all__ = ["sssp", "graphgen", "build"]
