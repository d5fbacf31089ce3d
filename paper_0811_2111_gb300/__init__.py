"""GB300-native checkerboard Metropolis engine for the 2-d XY model.

The compute path is the CUDA library ``libxy.so`` (C ABI in ``include/xy.h``);
this package holds its ctypes binding (``_lib``, same names as the C entry
points), a small torch-backed front end (``lattice``), the build script
(``build``) and the seeded workload definitions (``workloads``).
"""
