"""B300-native PVR hot path (patch-to-volume reconstruction, arXiv:1611.07289).

Submodules:
  pvr    -- Python binding of the C-ABI library libpvr.so (CUDA kernels, sm_103a)
  synth  -- seeded synthetic inputs (phantoms, stacks, motion)
Importing the package loads nothing; ``from paper_1611_07289_b300 import pvr``
loads the native library and fails loudly when it is missing.
"""
