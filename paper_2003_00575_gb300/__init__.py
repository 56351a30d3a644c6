"""GB300-native (sm_103a) hot path of FLIC (Fast Lidar Image Clustering, arXiv 2003.00575).

Submodules:
  flic   ctypes binding of libflic (the C ABI in include/flic.h); loads the CUDA library
  synth  seeded synthetic lidar frames (inputs only)

Importing the package loads nothing; ``paper_2003_00575_gb300.flic`` loads libflic.so and
fails loudly when it is missing.
"""
