// Solver kernels instantiated for RAPDB_FP8 storage.
#define RAPDB_ST RAPDB_FP8
#define RAPDB_SUF fp8
#include "kern_impl.cuh"
