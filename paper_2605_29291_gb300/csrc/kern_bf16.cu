// Solver kernels instantiated for RAPDB_BF16 storage.
#define RAPDB_ST RAPDB_BF16
#define RAPDB_SUF bf16
#include "kern_impl.cuh"
