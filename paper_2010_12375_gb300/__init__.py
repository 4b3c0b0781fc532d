"""GB300-native weakly-compressible SPH hot path (Riemann-solver WCSPH of SPHinXsys).

Submodules: `sph` (ctypes binding of libsph.so), `build` (nvcc build of the
library), `workloads` (seeded synthetic inputs). Importing the package loads
nothing; `sph.load()` loads the library and fails loudly if it is missing.
"""
