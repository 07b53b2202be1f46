// Launchers of the storage-templated solver kernels.  Each storage type
// (float32, bfloat16, FP8) is compiled in its own translation unit
// (kern_f32.cu, kern_bf16.cu, kern_fp8.cu) so that the builds run in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace rapdb_dev {

struct Inst;
struct State;
struct Ctrl;

// Coupling-pass tile variants picked by the autotuner:
//   RPW  rows streamed together by one warp (0: whole-row CTA stages),
//   UNR  16-byte chunks in flight per row and lane (register streaming),
//   NST  shared-memory slots (bulk-copy staging; 0 = registers),
//   CWB  bytes of each row per warp slot, or bytes per CTA stage (RPW = 0).
//   NST = -1: register streaming with the next batch's loads in flight.
//   RPW = 8 shares each 16-byte slice of x and v between eight rows, which
//   matters for FP8 (sixteen elements per slice); the float32 products of a
//   quantised matrix's refinement copy keep four rows per warp.
constexpr int NVAR = 10;
constexpr int kVarRPW[NVAR] = {4, 4, 4, 0, 0, 0, 4, 4, 8, 8};
constexpr int kVarUNR[NVAR] = {2, 4, 0, 0, 0, 0, 2, 4, 2, 1};
constexpr int kVarNST[NVAR] = {0, 0, 4, 3, 4, 3, -1, -1, 0, 0};
constexpr int kVarCWB[NVAR] = {0, 0, 512, 32768, 16384, 65536, 0, 0, 0, 0};

// dynamic shared memory of variant vi (8 warps).  Warp stages: mbarrier area
// rounded up to 128 bytes, then 8 * NST * RPW * CWB bytes of slots.  CTA
// stages: 128 bytes of mbarriers, 1 KB of row sums, NST * CWB bytes of slots.
inline size_t var_smem(int vi) {
  if (kVarNST[vi] <= 0) return 0;
  if (kVarRPW[vi] == 0) return (size_t)128 + 1024 + (size_t)kVarNST[vi] * kVarCWB[vi];
  const size_t bars = ((size_t)8 * kVarNST[vi] * 8 + 127) / 128 * 128;
  return bars + (size_t)8 * kVarNST[vi] * kVarRPW[vi] * kVarCWB[vi];
}

#define RAPDB_DECLARE_LAUNCHERS(SUF)                                                                              \
  cudaError_t prepare_##SUF();                                                                                    \
  void launch_vec_##SUF(dim3 g, size_t smem, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* vm,    \
                        float* XS, float* VS);                                                                    \
  void launch_pass_##SUF(int vi, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* pm,         \
                         const float* XS, const float* VS);                                                       \
  void launch_plain_##SUF(int vi, dim3 g, cudaStream_t s, const Inst* I, const float* x, const float* v,          \
                          const float* XS, const float* VS, const float* uold, float* U, float* W, double* part,  \
                          int level, const float* xlo, float* Ulo, int* err);                                     \
  void launch_pass_sym_##SUF(dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* pm,             \
                             const float* XS, const float* VS);                                                   \
  int pass_sym_occupancy_##SUF();

RAPDB_DECLARE_LAUNCHERS(f32)
RAPDB_DECLARE_LAUNCHERS(bf16)
RAPDB_DECLARE_LAUNCHERS(fp8)

}  // namespace rapdb_dev
