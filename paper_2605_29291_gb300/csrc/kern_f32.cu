// Solver kernels instantiated for RAPDB_F32 storage.
#define RAPDB_ST RAPDB_F32
#define RAPDB_SUF f32
#include "kern_impl.cuh"
