"""GB300-native batched growth step of planar vine robots (arXiv 2509.15180).

Submodules:
  vine    -- thin ctypes binding over the C-ABI library ``libvine.so``
             (loads the CUDA library on import and fails loudly without it)
  scenes  -- seeded synthetic inputs shaped like the paper's workloads
  build   -- compiles the CUDA library for sm_103a
"""
__all__ = ["vine", "scenes", "build"]
