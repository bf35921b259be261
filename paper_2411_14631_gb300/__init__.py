"""GB300-native AMR Godunov hydrodynamics: the data-parallel hot path of RAMSES
(arXiv 2411.14631, Table 1: godunov_fine / newdt_fine) as hand-written sm_103a CUDA
kernels behind a small C ABI."""
