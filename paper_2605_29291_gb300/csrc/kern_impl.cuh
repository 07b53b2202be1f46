// Launcher definitions for one storage type; included by kern_f32.cu,
// kern_bf16.cu and kern_fp8.cu with RAPDB_ST / RAPDB_SUF set.
#include "rapdb_kernels.cuh"
#include "rapdb_launch.h"

namespace rapdb_dev {

#define RAPDB_CAT2(a, b) a##b
#define RAPDB_CAT(a, b) RAPDB_CAT2(a, b)

static_assert(NWARP == 8, "var_smem assumes 8 warps per CTA");
static_assert(tma_smem_bytes<4, 4, 1024>() == 256 + 8 * 4 * 4 * 1024, "smem layout");
static_assert(tma_smem_bytes<3, 0, 32768>() == 128 + 1024 + 3 * 32768, "smem layout");

// Opt every bulk-copy variant in to its dynamic shared memory size.
cudaError_t RAPDB_CAT(prepare_, RAPDB_SUF)() {
  cudaError_t e = cudaSuccess;
#define RAPDB_ATTR(K, B)                                                                       \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(B));
  RAPDB_ATTR((k_pass<RAPDB_ST, 4, 0, 4, 512>), (tma_smem_bytes<4, 4, 512>()))
  RAPDB_ATTR((k_pass<RAPDB_ST, 0, 0, 3, 32768>), (tma_smem_bytes<3, 0, 32768>()))
  RAPDB_ATTR((k_pass<RAPDB_ST, 0, 0, 4, 16384>), (tma_smem_bytes<4, 0, 16384>()))
  RAPDB_ATTR((k_pass<RAPDB_ST, 0, 0, 3, 65536>), (tma_smem_bytes<3, 0, 65536>()))
  RAPDB_ATTR((k_pass_plain<RAPDB_ST, 4, 0, 4, 512>), (tma_smem_bytes<4, 4, 512>()))
  RAPDB_ATTR((k_pass_plain<RAPDB_ST, 0, 0, 3, 32768>), (tma_smem_bytes<3, 0, 32768>()))
  RAPDB_ATTR((k_pass_plain<RAPDB_ST, 0, 0, 4, 16384>), (tma_smem_bytes<4, 0, 16384>()))
  RAPDB_ATTR((k_pass_plain<RAPDB_ST, 0, 0, 3, 65536>), (tma_smem_bytes<3, 0, 65536>()))
#undef RAPDB_ATTR
  return e;
}

void RAPDB_CAT(launch_vec_, RAPDB_SUF)(dim3 g, size_t smem, cudaStream_t s, const Inst* I, State* S, Ctrl* C,
                                       const int* vm, float* XS, float* VS) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_vec<RAPDB_ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_vec<RAPDB_ST><<<g, NT, smem, s>>>(I, S, C, vm, XS, VS);
}

void RAPDB_CAT(launch_pass_, RAPDB_SUF)(int vi, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C,
                                        const int* pm, const float* XS, const float* VS) {
  switch (vi) {
    case 1: k_pass<RAPDB_ST, 4, 4, 0, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
    case 2: k_pass<RAPDB_ST, 4, 0, 4, 512><<<g, NT, var_smem(2), s>>>(I, S, C, pm, XS, VS); break;
    case 3: k_pass<RAPDB_ST, 0, 0, 3, 32768><<<g, NT, var_smem(3), s>>>(I, S, C, pm, XS, VS); break;
    case 4: k_pass<RAPDB_ST, 0, 0, 4, 16384><<<g, NT, var_smem(4), s>>>(I, S, C, pm, XS, VS); break;
    case 5: k_pass<RAPDB_ST, 0, 0, 3, 65536><<<g, NT, var_smem(5), s>>>(I, S, C, pm, XS, VS); break;
    case 6: k_pass<RAPDB_ST, 4, 2, -1, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
    case 7: k_pass<RAPDB_ST, 4, 4, -1, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
    case 8: k_pass<RAPDB_ST, 8, 2, 0, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
    case 9: k_pass<RAPDB_ST, 8, 1, 0, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
    default: k_pass<RAPDB_ST, 4, 2, 0, 0><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS); break;
  }
}

// The coupling pass of a context with symmetric block packing, and its CTAs
// resident per SM (the packed pass runs one persistent wave).
void RAPDB_CAT(launch_pass_sym_, RAPDB_SUF)(dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C,
                                            const int* pm, const float* XS, const float* VS) {
  k_pass_sym<RAPDB_ST><<<g, NT, 0, s>>>(I, S, C, pm, XS, VS);
}
int RAPDB_CAT(pass_sym_occupancy_, RAPDB_SUF)() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pass_sym<RAPDB_ST>, NT, 0) != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

void RAPDB_CAT(launch_plain_, RAPDB_SUF)(int vi, dim3 g, cudaStream_t s, const Inst* I, const float* x,
                                         const float* v, const float* XS, const float* VS, const float* uold,
                                         float* U, float* W, double* part, int level, const float* xlo,
                                         float* Ulo, int* err) {
  switch (vi) {
    case 1: k_pass_plain<RAPDB_ST, 4, 4, 0, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 2: k_pass_plain<RAPDB_ST, 4, 0, 4, 512><<<g, NT, var_smem(2), s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 3: k_pass_plain<RAPDB_ST, 0, 0, 3, 32768><<<g, NT, var_smem(3), s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 4: k_pass_plain<RAPDB_ST, 0, 0, 4, 16384><<<g, NT, var_smem(4), s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 5: k_pass_plain<RAPDB_ST, 0, 0, 3, 65536><<<g, NT, var_smem(5), s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 6: k_pass_plain<RAPDB_ST, 4, 2, -1, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 7: k_pass_plain<RAPDB_ST, 4, 4, -1, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 8: k_pass_plain<RAPDB_ST, 8, 2, 0, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    case 9: k_pass_plain<RAPDB_ST, 8, 1, 0, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
    default: k_pass_plain<RAPDB_ST, 4, 2, 0, 0><<<g, NT, 0, s>>>(I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err); break;
  }
}

}  // namespace rapdb_dev
