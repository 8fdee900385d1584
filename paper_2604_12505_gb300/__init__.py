"""GB300-native SPH fuel-sloshing simulator and LPV surrogate.

Submodules:
  sph        -- simulator front end over the CUDA library (include/sph.h)
  workloads  -- tank configurations and seeded synthetic inputs
  build      -- in-tree nvcc build of the CUDA library for sm_103a
"""
