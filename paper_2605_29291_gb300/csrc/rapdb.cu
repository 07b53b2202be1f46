// Host side of the C ABI declared in include/rapdb.h: context set-up, the
// graph-driven device loop, the stand-alone pass / KKT entry points,
// batched contexts and checkpointing.
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rapdb_launch.h"
#include "rapdb_util.cuh"

using namespace rapdb_dev;

namespace {

thread_local std::string g_last_error;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

struct InstHost {
  Inst I;                      // device-pointer copy uploaded to the context's array
  int64_t q_bytes;             // bytes of stored Q read by one pass
  int64_t qp_bytes = 0;        // bytes of the packed tiles read by one packed pass
  int64_t qpq_bytes = 0;       // ... of the quantised packed tiles (+ FP8 row scales)
};

}  // namespace

struct rapdb_ctx {
  int B = 1;
  bool batched = false;
  int mapped = 0;              // instances that have CTAs in the current block maps
  rapdb_params p{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used for graph capture
  int storage = RAPDB_F32;
  int variant = RAPDB_YX;
  std::vector<InstHost> hi;
  Inst* d_inst = nullptr;
  State* d_state = nullptr;
  Ctrl* d_ctrl = nullptr;
  int* d_vmap = nullptr;
  int* d_pmap = nullptr;
  int* d_flags = nullptr;
  int nvblk = 0, npblk = 0;
  size_t smem_vec = 0;
  float* XS = nullptr;
  float* VS = nullptr;
  // stand-alone scratch (single instance)
  float* tU = nullptr;
  float* tW = nullptr;
  float* tUo = nullptr;
  float* txv = nullptr;
  double* tpart = nullptr;
  double* tvpart = nullptr;
  double* tdots = nullptr;
  double* ty = nullptr;
  double* tg = nullptr;
  double* tout = nullptr;
  std::vector<void*> owned;
  cudaGraphExec_t gexec = nullptr;
  int g_bodies = 0;
  int64_t launches = 0;        // kernels launched by the current call
  int pvar = 0;                // coupling-pass tile variant (kVarRPW / kVarUNR)
  bool hyp = false;            // primal set with a hyperplane (two more kernels per body)
  int sym_grid = 0;            // pack_sym: CTAs of the row-streaming pass kernel (one resident wave)
  int sym_tile_grid = 0;       // ... and of the packed tile kernels (one CTA per SM)
  float tune_ms = 0.0f;        // autotuner: best pass time
  State* h_state = nullptr;    // pinned
  Ctrl* h_ctrl = nullptr;      // pinned, 2 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  std::string err;
  bool have_state = false;     // a solve finished (or set_state ran): checkpoint is valid
  // logging
  int log_cap = 0;
  double* tau_log = nullptr;
  double* kkt_log = nullptr;
  double* gap_log = nullptr;
  double* obj_log = nullptr;
  double* infeas_log = nullptr;
  int* trials_log = nullptr;
  float* x_log = nullptr;
  float* y_log = nullptr;
};

namespace {

// Storage-dispatching launchers (the kernels live in kern_{f32,bf16,fp8}.cu).
void launch_vec(int storage, dim3 g, size_t smem, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* vm,
                float* XS, float* VS) {
  if (storage == RAPDB_F32) launch_vec_f32(g, smem, s, I, S, C, vm, XS, VS);
  else if (storage == RAPDB_BF16) launch_vec_bf16(g, smem, s, I, S, C, vm, XS, VS);
  else launch_vec_fp8(g, smem, s, I, S, C, vm, XS, VS);
}

void launch_pass_sym(int storage, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* pm,
                     const float* XS, const float* VS) {
  if (storage == RAPDB_F32) launch_pass_sym_f32(g, s, I, S, C, pm, XS, VS);
  else if (storage == RAPDB_BF16) launch_pass_sym_bf16(g, s, I, S, C, pm, XS, VS);
  else launch_pass_sym_fp8(g, s, I, S, C, pm, XS, VS);
}

int pass_sym_occupancy(int storage) {
  if (storage == RAPDB_F32) return pass_sym_occupancy_f32();
  if (storage == RAPDB_BF16) return pass_sym_occupancy_bf16();
  return pass_sym_occupancy_fp8();
}

void launch_pass(int storage, int vi, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const int* pm,
                 const float* XS, const float* VS) {
  if (storage == RAPDB_F32) launch_pass_f32(vi, g, s, I, S, C, pm, XS, VS);
  else if (storage == RAPDB_BF16) launch_pass_bf16(vi, g, s, I, S, C, pm, XS, VS);
  else launch_pass_fp8(vi, g, s, I, S, C, pm, XS, VS);
}

void launch_plain(int storage, int vi, dim3 g, cudaStream_t s, const Inst* I, const float* x, const float* v,
                  const float* XS, const float* VS, const float* uold, float* U, float* W, double* part, int level,
                  int* err, const float* xlo = nullptr, float* Ulo = nullptr) {
  if (storage == RAPDB_F32) launch_plain_f32(vi, g, s, I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err);
  else if (storage == RAPDB_BF16) launch_plain_bf16(vi, g, s, I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err);
  else launch_plain_fp8(vi, g, s, I, x, v, XS, VS, uold, U, W, part, level, xlo, Ulo, err);
}

// The packed tile kernels of a context's storage (the float32 tiles serve
// every storage; the storage's own tiles serve the quantised level).
void launch_sym_tiles(int storage, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C, const float* VS) {
  if (storage == RAPDB_BF16) k_sym_tiles<RAPDB_BF16><<<g, NTS, sym_smem_bytes(), s>>>(I, S, C, VS);
  else if (storage == RAPDB_FP8) k_sym_tiles<RAPDB_FP8><<<g, NTS, sym_smem_bytes(), s>>>(I, S, C, VS);
  else k_sym_tiles<RAPDB_F32><<<g, NTS, sym_smem_bytes(), s>>>(I, S, C, VS);
}
void launch_sym_finish(int storage, dim3 g, cudaStream_t s, const Inst* I, State* S, Ctrl* C) {
  if (storage == RAPDB_BF16) k_sym_finish<RAPDB_BF16><<<g, NT, 0, s>>>(I, S, C);
  else if (storage == RAPDB_FP8) k_sym_finish<RAPDB_FP8><<<g, NT, 0, s>>>(I, S, C);
  else k_sym_finish<RAPDB_F32><<<g, NT, 0, s>>>(I, S, C);
}
// The pieces of v for the quantised tiles (before launch_sym_plain with quant).
void launch_sym_pieces(int storage, cudaStream_t s, const Inst* I, const float* v) {
  if (storage == RAPDB_BF16) k_sym_pieces<RAPDB_BF16><<<128, NT, 0, s>>>(I, v);
  else if (storage == RAPDB_FP8) k_sym_pieces<RAPDB_FP8><<<128, NT, 0, s>>>(I, v);
}
void launch_sym_plain(int storage, dim3 g, cudaStream_t s, const Inst* I, const float* v, int quant, int* err) {
  if (storage == RAPDB_BF16) k_sym_plain<RAPDB_BF16><<<g, NTS, sym_smem_bytes(), s>>>(I, v, quant, err);
  else if (storage == RAPDB_FP8) k_sym_plain<RAPDB_FP8><<<g, NTS, sym_smem_bytes(), s>>>(I, v, quant, err);
  else k_sym_plain<RAPDB_F32><<<g, NTS, sym_smem_bytes(), s>>>(I, v, 0, err);
}

// NVTX range for the duration of a scope (set-up, solve, stand-alone pass
// and residual phases show up by name in a profiler's timeline; no cost
// without one attached).
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
};

std::string ctrl_error_text(int code) {
  if (code == 1) return "a bounded wait in the coupling pass gave up";
  return "range check " + std::to_string(code) + " of the checked build failed";
}

rapdb_status fail(rapdb_ctx* ctx, rapdb_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  g_last_error = msg;
  return st;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? RAPDB_ERR_NOMEM : RAPDB_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                            \
    }                                                                                             \
  } while (0)

template <typename T>
rapdb_status dalloc(rapdb_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess)
    return fail(ctx, e == cudaErrorMemoryAllocation ? RAPDB_ERR_NOMEM : RAPDB_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  ctx->owned.push_back(q);
  e = cudaMemsetAsync(q, 0, bytes, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, RAPDB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  *p = (T*)q;
  return RAPDB_OK;
}

#define AL(ptr, count)                                     \
  do {                                                     \
    rapdb_status s_ = dalloc(ctx, &(ptr), (size_t)(count)); \
    if (s_ != RAPDB_OK) return s_;                         \
  } while (0)

int pick_rows_per_block(int64_t n, int64_t M) {
  // starting tile (and the batched default): 32 rows, one 4-row group per
  // warp; the autotuner widens it for large single instances
  (void)n;
  (void)M;
  return 32;
}

DevParams make_devparams(const rapdb_params& p, const rapdb_ctx* ctx) {
  DevParams d{};
  d.variant = p.variant;
  d.c_nm = p.c_nm;
  d.backtracking = p.backtracking;
  d.restart = p.restart;
  d.restart_period = p.restart_period;
  d.restart_from_average = p.restart_from_average;
  d.max_iter = p.max_iter;
  d.max_trials = p.max_trials;
  d.kkt_every = p.kkt_every;
  d.refine = p.refine;
  d.gap_first = p.gap_first;
  d.gap_every = p.gap_every;
  d.gap_inner_max = p.gap_inner_max;
  d.dual_simplex = p.dual_set == RAPDB_DUAL_SIMPLEX ? 1 : 0;
  d.warm_tau = p.restart_warm_tau ? 1 : 0;
  d.dual_r = p.dual_radius;
  d.mu = p.mu;
  d.c_alpha = p.c_alpha;
  d.c_beta = p.c_beta;
  d.delta = p.delta;
  d.eta = p.eta;
  d.tau_bar = p.tau_bar;
  d.gamma0 = p.gamma0;
  d.tol = p.tol;
  d.stall_ratio = p.stall_ratio;
  d.xi = p.xi;
  d.q = p.q;
  d.log_cap = ctx->log_cap;
  d.tau_log = ctx->tau_log;
  d.kkt_log = ctx->kkt_log;
  d.gap_log = ctx->gap_log;
  d.obj_log = ctx->obj_log;
  d.infeas_log = ctx->infeas_log;
  d.trials_log = ctx->trials_log;
  d.x_log = ctx->x_log;
  d.y_log = ctx->y_log;
  return d;
}

rapdb_status check_params(rapdb_ctx* ctx, const rapdb_params* p) {
  if (!p) return fail(ctx, RAPDB_ERR_INVALID, "params is NULL");
  if (p->variant != RAPDB_YX && p->variant != RAPDB_XY) return fail(ctx, RAPDB_ERR_INVALID, "bad variant");
  if (p->storage < RAPDB_F32 || p->storage > RAPDB_FP8) return fail(ctx, RAPDB_ERR_INVALID, "bad storage");
  if (p->restart < RAPDB_RESTART_NONE || p->restart > RAPDB_RESTART_GAP)
    return fail(ctx, RAPDB_ERR_INVALID, "bad restart mode");
  if (p->restart == RAPDB_RESTART_GAP &&
      (p->restart_from_average || !(p->xi > 0.0) || !(p->q > 0.0) || p->gap_first < 0 || p->gap_every < 1 ||
       p->gap_inner_max < 1))
    return fail(ctx, RAPDB_ERR_INVALID,
                "adaptive restart needs xi > 0, q > 0, gap_first >= 0, gap_every >= 1, gap_inner_max >= 1 and "
                "restarts from the last iterate");
  if (p->restart == RAPDB_RESTART_FIXED && p->restart_period < 1)
    return fail(ctx, RAPDB_ERR_INVALID, "restart_period must be >= 1");
  if (!(p->eta > 0.0 && p->eta < 1.0)) return fail(ctx, RAPDB_ERR_INVALID, "eta must be in (0,1)");
  if (!(p->tau_bar > 0.0) || !(p->gamma0 > 0.0)) return fail(ctx, RAPDB_ERR_INVALID, "tau_bar, gamma0 must be > 0");
  if (!(p->c_alpha > 0.0) || p->mu < 0.0) return fail(ctx, RAPDB_ERR_INVALID, "c_alpha > 0, mu >= 0 required");
  if (p->variant == RAPDB_XY && !(p->c_beta >= 0.0)) return fail(ctx, RAPDB_ERR_INVALID, "c_beta >= 0 required");
  if (p->max_iter < 0 || p->max_trials < 1) return fail(ctx, RAPDB_ERR_INVALID, "max_iter >= 0, max_trials >= 1");
  if (p->rows_per_block < 0 || (p->rows_per_block % 32) != 0)
    return fail(ctx, RAPDB_ERR_INVALID, "rows_per_block must be 0 (auto) or a multiple of 32");
  if (p->rows_per_block > 0 && (p->pass_variant < 0 || p->pass_variant >= NVAR))
    return fail(ctx, RAPDB_ERR_INVALID, "pass_variant out of range");
  if (p->dual_set != RAPDB_DUAL_NONNEG && p->dual_set != RAPDB_DUAL_SIMPLEX)
    return fail(ctx, RAPDB_ERR_INVALID, "dual_set must be RAPDB_DUAL_NONNEG or RAPDB_DUAL_SIMPLEX");
  if (p->dual_set == RAPDB_DUAL_SIMPLEX && !(p->dual_radius > 0.0 && std::isfinite(p->dual_radius)))
    return fail(ctx, RAPDB_ERR_INVALID, "dual_radius must be positive and finite");
  if (p->pack_sym != 0 && p->pack_sym != 1) return fail(ctx, RAPDB_ERR_INVALID, "pack_sym must be 0 or 1");
  if (p->pack_sym && !p->refine)
    return fail(ctx, RAPDB_ERR_INVALID,
                "pack_sym packs the float32 matrices of the compensated trial passes: it needs refine = 1");
  return RAPDB_OK;
}

// Build one instance's buffers.  Q, c, d, lb, ub, q0diag are the caller's device arrays.
rapdb_status build_instance(rapdb_ctx* ctx, InstHost& H, int64_t n64, int64_t m64, int q0_kind, const float* Q,
                            const float* q0diag, const float* c, const float* d, const float* lb, const float* ub,
                            int rb_override, int64_t p_eq = 0, const float* A_eq = nullptr,
                            const float* b_eq = nullptr, const float* hyp_a = nullptr, double hyp_beta = 0.0) {
  const rapdb_params& p = ctx->p;
  // inequalities 1..m_in with stored matrices, then p_eq linear equalities
  const int n = (int)n64, m_in = (int)m64, pe = (int)p_eq, m = m_in + pe;
  const int M = (q0_kind == RAPDB_Q0_DENSE) ? m_in + 1 : m_in;
  Inst& I = H.I;
  I = Inst{};
  I.n = n;
  I.m = m;
  I.m_ineq = m_in;
  I.M = M;
  I.q0_kind = q0_kind;
  I.s_off = (q0_kind == RAPDB_Q0_DENSE) ? 0 : 1;
  I.storage = p.storage;
  I.ldv = (int)round_up(n, 16);
  const int ldv = I.ldv;
  cudaStream_t st = ctx->stream;

  // validation
  CK(cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), st));
  k_validate<<<1024, 256, 0, st>>>(Q, n, M, c, m_in, d, lb, ub, q0_kind == RAPDB_Q0_DIAG ? q0diag : nullptr,
                                   ctx->d_flags);
  CK(cudaGetLastError());
  int flags[4];
  CK(cudaMemcpyAsync(flags, ctx->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flags[0]) return fail(ctx, RAPDB_ERR_INVALID, "NaN or Inf in the problem data");
  if (flags[1]) return fail(ctx, RAPDB_ERR_INVALID, "negative diagonal entry: some Q_i is not PSD");
  if (flags[2]) return fail(ctx, RAPDB_ERR_INVALID, "lb > ub");
  std::vector<float> hb(pe);
  if (pe > 0) {
    std::vector<float> ha((size_t)pe * n);
    CK(cudaMemcpy(ha.data(), A_eq, ha.size() * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hb.data(), b_eq, (size_t)pe * 4, cudaMemcpyDeviceToHost));
    for (float v : ha)
      if (!std::isfinite(v)) return fail(ctx, RAPDB_ERR_INVALID, "NaN or Inf in the equality data");
    for (float v : hb)
      if (!std::isfinite(v)) return fail(ctx, RAPDB_ERR_INVALID, "NaN or Inf in the equality data");
  }

  // stored Q
  const bool aligned = ((uintptr_t)Q % 16) == 0;
  const int64_t rows = (int64_t)M * n;
  if (p.storage == RAPDB_F32) {
    if (n % 4 == 0 && aligned) {
      I.Q = Q;
      I.ld = n;
    } else {
      I.ld = (int)round_up(n, 4);
      float* q = nullptr;
      AL(q, rows * I.ld);
      if (rows > 0)
        CK(cudaMemcpy2DAsync(q, (size_t)I.ld * 4, Q, (size_t)n * 4, (size_t)n * 4, (size_t)rows,
                             cudaMemcpyDeviceToDevice, st));
      I.Q = q;
    }
    H.q_bytes = rows * (int64_t)I.ld * 4;
  } else {
    const int EB = (p.storage == RAPDB_BF16) ? 2 : 1;
    I.ld = (int)round_up(n, 16 / EB);
    uint8_t* q = nullptr;
    AL(q, rows * I.ld * EB);
    if (p.storage == RAPDB_BF16) {
      if (rows > 0) k_quant_bf16<<<4096, 256, 0, st>>>(Q, n, rows, I.ld, (__nv_bfloat16*)q);
    } else {
      float *rinv = nullptr, *scale = nullptr;
      AL(rinv, (size_t)std::max(M, 1) * ldv);
      AL(scale, (size_t)std::max(M, 1) * ldv);
      if (rows > 0) {
        k_fp8_scales<<<256, 256, 0, st>>>(Q, n, M, ldv, rinv, scale);
        k_quant_fp8<<<4096, 256, 0, st>>>(Q, n, M, I.ld, ldv, rinv, (__nv_fp8_storage_t*)q);
      }
      I.qscale = scale;
    }
    CK(cudaGetLastError());
    I.Q = q;
    H.q_bytes = rows * (int64_t)I.ld * EB;
    if (p.refine) {
      if (n % 4 == 0 && aligned) {
        I.Q32 = Q;
        I.ld32 = n;
      } else {
        I.ld32 = (int)round_up(n, 4);
        float* q32 = nullptr;
        AL(q32, rows * I.ld32);
        if (rows > 0)
          CK(cudaMemcpy2DAsync(q32, (size_t)I.ld32 * 4, Q, (size_t)n * 4, (size_t)n * 4, (size_t)rows,
                               cudaMemcpyDeviceToDevice, st));
        I.Q32 = q32;
      }
    }
  }

  // vectors (padded to ldv; padding zero)
  float *cc = nullptr, *lbp = nullptr, *ubp = nullptr, *q0d = nullptr;
  double* dd = nullptr;
  AL(cc, (size_t)(m + 1) * ldv);
  CK(cudaMemcpy2DAsync(cc, (size_t)ldv * 4, c, (size_t)n * 4, (size_t)n * 4, (size_t)(m_in + 1),
                       cudaMemcpyDeviceToDevice, st));
  if (pe > 0)   // equality rows a_k after the inequality rows
    CK(cudaMemcpy2DAsync(cc + (size_t)(m_in + 1) * ldv, (size_t)ldv * 4, A_eq, (size_t)n * 4, (size_t)n * 4,
                         (size_t)pe, cudaMemcpyDeviceToDevice, st));
  AL(lbp, ldv);
  AL(ubp, ldv);
  CK(cudaMemcpyAsync(lbp, lb, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(ubp, ub, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
  AL(q0d, ldv);
  if (q0_kind == RAPDB_Q0_DIAG) CK(cudaMemcpyAsync(q0d, q0diag, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
  AL(dd, std::max(m, 1));
  double dn = 0.0;
  if (m_in > 0) {
    k_f2d<<<1, 256, 0, st>>>(d, dd, m_in);
    std::vector<float> hd(m_in);
    CK(cudaMemcpyAsync(hd.data(), d, (size_t)m_in * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < m_in; ++i) dn += (double)hd[i] * (double)hd[i];
  }
  if (pe > 0) {   // an equality a'x = b is the constraint a'x - b: d = -b
    std::vector<double> hdb(pe);
    for (int k = 0; k < pe; ++k) {
      hdb[k] = -(double)hb[k];
      dn += hdb[k] * hdb[k];
    }
    CK(cudaMemcpy(dd + m_in, hdb.data(), (size_t)pe * 8, cudaMemcpyHostToDevice));
  }
  I.c = cc;
  I.lb = lbp;
  I.ub = ubp;
  I.q0diag = q0d;
  if (hyp_a) {
    // primal set X = box with {a'x = beta}: a (padded with zeros), and the
    // projection's and the cone residual's per-column pairs
    std::vector<float> ha(n);
    CK(cudaMemcpy(ha.data(), hyp_a, (size_t)n * 4, cudaMemcpyDeviceToHost));
    bool any = false;
    for (float v : ha) {
      if (!std::isfinite(v)) return fail(ctx, RAPDB_ERR_INVALID, "NaN or Inf in the hyperplane of X");
      any = any || v != 0.0f;
    }
    if (!any || !std::isfinite(hyp_beta)) return fail(ctx, RAPDB_ERR_INVALID, "the hyperplane of X is degenerate");
    float* da = nullptr;
    AL(da, ldv);
    CK(cudaMemcpyAsync(da, hyp_a, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    I.hyp_a = da;
    I.hyp_beta = hyp_beta;
    float2* hv = nullptr;
    float2* hg = nullptr;
    AL(hv, ldv);
    AL(hg, ldv);
    I.hv = hv;
    I.hg = hg;
  }
  I.dcon = dd;
  I.dnorm = sqrt(dn);

  // tiles
  // (a context with packed tiles runs its row-streaming passes on 64-row items)
  I.rb = p.pack_sym ? 64 : (rb_override > 0 ? rb_override : pick_rows_per_block(n, M));
  I.nrb = (n + I.rb - 1) / I.rb;
  I.ncb = (n + VCOL - 1) / VCOL;

  // solver buffers
  const int mm = std::max(m, 1);
  for (int s = 0; s < 2; ++s) {
    AL(I.xb[s], ldv);
    AL(I.xf[s], ldv);
    AL(I.xl[s], ldv);
    if (p.refine) AL(I.Ulo[s], (size_t)(m + 1) * ldv);
    AL(I.yb[s], mm);
    AL(I.U[s], (size_t)(m + 1) * ldv);
    AL(I.gb[s], mm);
    if (p.variant == RAPDB_XY) AL(I.gx[s], ldv);
  }
  AL(I.W, (size_t)(m + 1) * ldv);
  AL(I.dv, ldv);
  AL(I.gnew, mm);
  AL(I.part, (size_t)std::max(M, 1) * NDOT * I.nrb);
  AL(I.mcount, std::max(M, 1));
  AL(I.vpart, (size_t)I.ncb * NVP);
  AL(I.dots, (size_t)(m + 1) * NDOT);
  if (p.restart_from_average) {
    AL(I.xcum, ldv);
    AL(I.ycum, mm);
  }
  if (p.restart == RAPDB_RESTART_GAP) {
    AL(I.gz, ldv);
    AL(I.gzf, ldv);
    AL(I.gwf, ldv);
    AL(I.gpf, ldv);
  }
  if (p.pack_sym && M > 0) {
    // symmetric block packing of the float32 matrices the trial passes read
    const float* Qf = (p.storage == RAPDB_F32) ? (const float*)I.Q : I.Q32;
    const int ldq = (p.storage == RAPDB_F32) ? I.ld : I.ld32;
    CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), st));
    k_sym_check<<<2048, dim3(32, 8), 0, st>>>(Qf, ldq, n, M, ctx->d_flags);
    CK(cudaGetLastError());
    int asym = 0;
    CK(cudaMemcpyAsync(&asym, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (asym) return fail(ctx, RAPDB_ERR_INVALID, "pack_sym needs exactly symmetric Q_i (Q_i[j][k] == Q_i[k][j])");
    const int T = (n + STB - 1) / STB;
    const int64_t ntile64 = (int64_t)T * (T + 1) / 2;
    if ((int64_t)M * ntile64 > (int64_t)INT32_MAX / 2)
      return fail(ctx, RAPDB_ERR_INVALID, "pack_sym: too many tiles for this n and m");
    const int ntile = (int)ntile64;
    std::vector<int> tij;
    tij.reserve(ntile);
    for (int a = 0; a < T; ++a)
      for (int b2 = a; b2 < T; ++b2) tij.push_back((a << 16) | b2);
    int* dtij = nullptr;
    float* qp = nullptr;
    AL(dtij, ntile);
    CK(cudaMemcpyAsync(dtij, tij.data(), tij.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    AL(qp, (size_t)M * ntile * STB * STB);
    k_pack_sym<<<4096, 256, 0, st>>>(Qf, ldq, n, M, T, ntile, dtij, qp);
    CK(cudaGetLastError());
    AL(I.sp, (size_t)2 * M * T * T * STB);     // two slot sets (two right-hand sides)
    AL(I.spart, (size_t)M * NDOT * T);
    I.Qp = qp;
    I.tij = dtij;
    I.tsym = T;
    I.ntile = ntile;
    H.qp_bytes = (int64_t)M * ntile * STB * STB * 4;
    if (p.storage != RAPDB_F32) {
      // the stored BF16 / FP8 codes in the same tiles: the trial passes of
      // the quantised level read these (a half / a quarter of the bytes)
      const int EB = (p.storage == RAPDB_BF16) ? 2 : 1;
      uint8_t* qq = nullptr;
      AL(qq, (size_t)M * ntile * STB * STB * EB);
      if (EB == 2)
        k_pack_sym_codes<uint16_t><<<4096, 256, 0, st>>>((const uint16_t*)I.Q, I.ld, n, M, ntile, dtij, (uint16_t*)qq);
      else
        k_pack_sym_codes<uint8_t><<<4096, 256, 0, st>>>((const uint8_t*)I.Q, I.ld, n, M, ntile, dtij, qq);
      CK(cudaGetLastError());
      I.Qpq = qq;
      H.qpq_bytes = (int64_t)M * ntile * STB * STB * EB + (EB == 1 ? (int64_t)M * n * 4 : 0);
      // the pieces of the trial right-hand side, one 2 KB (BF16) / 1 KB (FP8)
      // block per 128 entries; the rows past the pieces stay zero
      const size_t pqb = (size_t)(EB == 1 ? M : 1) * T * sym_piece_bytes(EB);
      AL(I.Pq, pqb);
      CK(cudaMemsetAsync(I.Pq, 0, pqb, st));
    }
  }
  I.P = make_devparams(p, ctx);
  return RAPDB_OK;
}

// Upload instance table + block maps, create the capture stream and graph.
rapdb_status finalize_ctx(rapdb_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int B = ctx->B;
  std::vector<int> vmap, pmap;
  int mmax = 1;
  for (int b = 0; b < B; ++b) {
    Inst& I = ctx->hi[b].I;
    I.vblk0 = (int)vmap.size();
    for (int k = 0; k < I.ncb; ++k) vmap.push_back(b);
    I.pblk0 = (int)pmap.size();
    for (int k = 0; k < I.M * I.nrb; ++k) pmap.push_back(b);
    mmax = std::max(mmax, I.m);
  }
  ctx->nvblk = (int)vmap.size();
  ctx->npblk = (int)pmap.size();
  ctx->mapped = B;
  ctx->smem_vec = (size_t)mmax * VEC_SMEM_PER_CON;
  if (mmax > RAPDB_MAX_CONSTRAINTS) return fail(ctx, RAPDB_ERR_INVALID, "too many constraints (m > 6400)");
  AL(ctx->d_vmap, vmap.size());
  AL(ctx->d_pmap, std::max<size_t>(pmap.size(), 1));
  CK(cudaMemcpyAsync(ctx->d_vmap, vmap.data(), vmap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!pmap.empty())
    CK(cudaMemcpyAsync(ctx->d_pmap, pmap.data(), pmap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  AL(ctx->d_inst, B);
  AL(ctx->d_state, B);
  AL(ctx->d_ctrl, 1);
  std::vector<Inst> tmp(B);
  for (int b = 0; b < B; ++b) tmp[b] = ctx->hi[b].I;
  CK(cudaMemcpyAsync(ctx->d_inst, tmp.data(), B * sizeof(Inst), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  CK(prepare_f32());
  CK(prepare_bf16());
  CK(prepare_fp8());
  CK(cudaMallocHost((void**)&ctx->h_state, sizeof(State) * B));
  CK(cudaMallocHost((void**)&ctx->h_ctrl, sizeof(Ctrl) * 2));
  CK(cudaEventCreateWithFlags(&ctx->ev[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev[1], cudaEventDisableTiming));
  CK(cudaEventCreate(&ctx->t0));
  CK(cudaEventCreate(&ctx->t1));
  CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
  return RAPDB_OK;
}

rapdb_status upload_params(rapdb_ctx* ctx) {
  std::vector<Inst> tmp(ctx->B);
  for (int b = 0; b < ctx->B; ++b) {
    ctx->hi[b].I.P = make_devparams(ctx->p, ctx);
    tmp[b] = ctx->hi[b].I;
  }
  CK(cudaMemcpyAsync(ctx->d_inst, tmp.data(), ctx->B * sizeof(Inst), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return RAPDB_OK;
}

// One body of the device loop on stream s.
rapdb_status launch_body(rapdb_ctx* ctx, cudaStream_t s) {
  const int st = ctx->storage;
  const dim3 gv(ctx->nvblk), gp(std::max(ctx->npblk, 1)), blk(NT);
  const size_t sm = ctx->smem_vec;
  (void)blk;
  auto vec = [&]() { launch_vec(st, gv, sm, s, ctx->d_inst, ctx->d_state, ctx->d_ctrl, ctx->d_vmap, ctx->XS, ctx->VS); };
  vec();
  if (ctx->hyp) {
    // X with a hyperplane: the projection's scalar, then x column by column
    k_hyp<0><<<1, NTH, 0, s>>>(ctx->d_inst, ctx->d_state);
    vec();
  }
  if (ctx->sym_grid > 0) {
    const Inst& I = ctx->hi[0].I;
    launch_pass_sym(st, dim3(ctx->sym_grid), s, ctx->d_inst, ctx->d_state, ctx->d_ctrl, ctx->d_pmap, ctx->XS,
                    ctx->VS);
    launch_sym_tiles(st, dim3(ctx->sym_tile_grid), s, ctx->d_inst, ctx->d_state, ctx->d_ctrl, ctx->VS);
    launch_sym_finish(st, dim3(I.M * I.tsym), s, ctx->d_inst, ctx->d_state, ctx->d_ctrl);
    k_sym_ctrl<0><<<1, NT, 0, s>>>(ctx->d_inst, ctx->d_state, ctx->d_ctrl);
  } else if (ctx->npblk > 0)
    launch_pass(st, ctx->pvar, gp, s, ctx->d_inst, ctx->d_state, ctx->d_ctrl, ctx->d_pmap, ctx->XS, ctx->VS);
  if (ctx->variant == RAPDB_XY) vec();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, RAPDB_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return RAPDB_OK;
}

rapdb_status build_graph(rapdb_ctx* ctx, int bodies) {
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < bodies; ++k) {
    rapdb_status s = launch_body(ctx, ctx->cap);
    if (s != RAPDB_OK) {
      cudaStreamEndCapture(ctx->cap, &g);
      if (g) cudaGraphDestroy(g);
      return s;
    }
  }
  CK(cudaStreamEndCapture(ctx->cap, &g));
  cudaError_t e = cudaGraphInstantiate(&ctx->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, RAPDB_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  ctx->g_bodies = bodies;
  return RAPDB_OK;
}

// Block maps over the instances still running (a batched context drops the
// finished ones, so that their CTAs are no longer launched only to exit);
// `run[b]` selects instance b.  Rebuilds the loop graph for the new grids.
// The caller has synchronised the stream.
rapdb_status set_block_maps(rapdb_ctx* ctx, const std::vector<char>& run) {
  cudaStream_t st = ctx->stream;
  std::vector<int> vmap, pmap;
  int nact = 0;
  for (int b = 0; b < ctx->B; ++b) {
    if (!run[b]) continue;
    Inst& I = ctx->hi[b].I;
    ++nact;
    I.vblk0 = (int)vmap.size();
    for (int k = 0; k < I.ncb; ++k) vmap.push_back(b);
    I.pblk0 = (int)pmap.size();
    for (int k = 0; k < I.M * I.nrb; ++k) pmap.push_back(b);
  }
  if (!vmap.empty())
    CK(cudaMemcpyAsync(ctx->d_vmap, vmap.data(), vmap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!pmap.empty())
    CK(cudaMemcpyAsync(ctx->d_pmap, pmap.data(), pmap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<Inst> tmp(ctx->B);
  for (int b = 0; b < ctx->B; ++b) tmp[b] = ctx->hi[b].I;
  CK(cudaMemcpyAsync(ctx->d_inst, tmp.data(), ctx->B * sizeof(Inst), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->nvblk = (int)vmap.size();
  ctx->npblk = (int)pmap.size();
  ctx->mapped = nact;
  if (ctx->p.use_graph && nact > 0) return build_graph(ctx, 32);
  return RAPDB_OK;
}

// Run the device loop until every instance is done.  The host never waits
// per trial: it keeps two graph launches (each `g_bodies` bodies) in flight
// and reads the 'active' counter of the older one.
rapdb_status run_loop(rapdb_ctx* ctx, int64_t max_bodies) {
  cudaStream_t st = ctx->stream;
  const bool graph = ctx->p.use_graph != 0;
  const int per = graph ? ctx->g_bodies : 16;
  int64_t launched = 0;
  int slot = 0, pending = 0;
  bool done = false;
  while (!done) {
    if (launched >= max_bodies) break;
    if (graph) {
      CK(cudaGraphLaunch(ctx->gexec, st));
    } else {
      for (int k = 0; k < per; ++k) {
        rapdb_status s = launch_body(ctx, st);
        if (s != RAPDB_OK) return s;
      }
    }
    launched += per;
    // kernels per body: vector, pass (xy: a second vector kernel), and the
    // packed tile, row-block and control kernels of a pack_sym context
    ctx->launches +=
        (int64_t)per * ((ctx->variant == RAPDB_XY ? 3 : 2) + (ctx->sym_grid > 0 ? 3 : 0) + (ctx->hyp ? 2 : 0));
    CK(cudaMemcpyAsync(&ctx->h_ctrl[slot], ctx->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ctx->ev[slot], st));
    pending++;
    if (pending == 2) {
      const int old = slot ^ 1;
      CK(cudaEventSynchronize(ctx->ev[old]));
      pending = 1;
      const int act = ctx->h_ctrl[old].active;
      if (act <= 0 || ctx->h_ctrl[old].err != 0) {
        done = true;     // all instances finished, or a kernel reported an error
      } else if (ctx->batched && 2 * act <= ctx->mapped && ctx->npblk > 4 * 152) {
        // half of the mapped instances have finished: launch CTAs for the
        // running ones only (each instance's arithmetic is unchanged)
        CK(cudaStreamSynchronize(st));
        CK(cudaMemcpy(ctx->h_state, ctx->d_state, sizeof(State) * ctx->B, cudaMemcpyDeviceToHost));
        std::vector<char> run(ctx->B);
        for (int b = 0; b < ctx->B; ++b) run[b] = ctx->h_state[b].phase != PH_DONE;
        rapdb_status s = set_block_maps(ctx, run);
        if (s != RAPDB_OK) return s;
        pending = 0;
      }
    }
    slot ^= 1;
  }
  CK(cudaStreamSynchronize(st));
  return RAPDB_OK;
}

// Re-tile instance 0 (single-instance contexts): rows per CTA and the pass
// block map.  Buffers were sized for the smallest tile (32 rows).
rapdb_status retile(rapdb_ctx* ctx, int rb) {
  cudaStream_t st = ctx->stream;
  Inst& I = ctx->hi[0].I;
  I.rb = rb;
  I.nrb = (I.n + rb - 1) / rb;
  ctx->npblk = I.M * I.nrb;
  std::vector<int> pmap((size_t)ctx->npblk, 0);
  CK(cudaMemcpyAsync(ctx->d_pmap, pmap.data(), pmap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return RAPDB_OK;
}

// Autotuner: time every (tile variant, rows per CTA) on the caller's data with
// CUDA events and keep the fastest.
rapdb_status autotune(rapdb_ctx* ctx) {
  NvtxScope nvtx_scope("rapdb_autotune");
  cudaStream_t st = ctx->stream;
  const Inst I0 = ctx->hi[0].I;
  const int rbs[3] = {32, 64, 128};
  const int64_t bytes = ctx->hi[0].q_bytes;
  const int reps = bytes > (int64_t)(256 << 20) ? 2 : 5;
  float best = 1e30f;
  int best_v = 0, best_rb = 32;
  for (int ri = 0; ri < 3; ++ri) {
    if (ri > 0 && rbs[ri] > 2 * I0.n) break;
    rapdb_status s = retile(ctx, rbs[ri]);
    if (s != RAPDB_OK) return s;
    const int grid = ctx->npblk;
    for (int vi = 0; vi < NVAR; ++vi) {
      const Inst& I = ctx->hi[0].I;
      // time the pass the solver's trials run: float32 storage with
      // refinement runs the incremental compensated pass (level 3) throughout
      const bool inc = I.storage == RAPDB_F32 && I.P.refine && I.Ulo[0] != nullptr;
      auto go = [&]() {
        if (inc)
          launch_plain(I.storage, vi, dim3(grid), st, ctx->d_inst, I.xf[0], I.dv, ctx->XS, ctx->VS, I.U[0], ctx->tU,
                       ctx->tW, ctx->tpart, 3, &ctx->d_ctrl->err, I.xl[0], ctx->tUo);
        else
          launch_plain(I.storage, vi, dim3(grid), st, ctx->d_inst, I.xf[0], I.dv, ctx->XS, ctx->VS, nullptr, ctx->tU,
                       ctx->tW, ctx->tpart, 0, &ctx->d_ctrl->err);
      };
      go();
      CK(cudaGetLastError());
      CK(cudaEventRecord(ctx->t0, st));
      for (int r = 0; r < reps; ++r) go();
      CK(cudaEventRecord(ctx->t1, st));
      CK(cudaEventSynchronize(ctx->t1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
      if (inc) {
        // the same tile also runs the two-right-hand-side passes of the
        // smoothed gap (a few percent of a solve): weigh them in lightly, so
        // that near-ties between tiles go to the one that does both well
        auto go0 = [&]() {
          launch_plain(I.storage, vi, dim3(grid), st, ctx->d_inst, I.xf[0], I.dv, ctx->XS, ctx->VS, nullptr,
                       ctx->tU, ctx->tW, ctx->tpart, 0, &ctx->d_ctrl->err);
        };
        go0();
        CK(cudaEventRecord(ctx->t0, st));
        for (int r = 0; r < reps; ++r) go0();
        CK(cudaEventRecord(ctx->t1, st));
        CK(cudaEventSynchronize(ctx->t1));
        float ms0 = 0.0f;
        CK(cudaEventElapsedTime(&ms0, ctx->t0, ctx->t1));
        ms += 0.1f * ms0;
      }
      if (ms < best) {
        best = ms;
        best_v = vi;
        best_rb = rbs[ri];
      }
    }
  }
  ctx->pvar = best_v;
  ctx->tune_ms = best / reps;      // (includes the 0.1 weight of the two-RHS pass when incremental)
  return retile(ctx, best_rb);
}

// Tiles found by the autotuner, remembered per device and problem shape so
// that later contexts of the same shape skip the timing launches.  Key:
// device, n, stored matrices, storage, incremental (float32 with refinement),
// row stride, Q_0 kind.
using TileKey = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tile_mutex;
std::map<TileKey, std::pair<int, int>> g_tile_cache;   // -> (variant, rows per block)

TileKey tile_key(const rapdb_ctx* ctx) {
  const Inst& I = ctx->hi[0].I;
  int dev = 0;
  cudaGetDevice(&dev);
  const int inc = (I.storage == RAPDB_F32 && I.P.refine && I.Ulo[0]) ? 1 : 0;
  return TileKey(dev, I.n, I.M, I.storage, inc, I.ld, I.q0_kind);
}

// Autotune, or take the tile a previous context of the same shape found.
rapdb_status pick_tile(rapdb_ctx* ctx) {
  const TileKey key = tile_key(ctx);
  {
    std::lock_guard<std::mutex> lk(g_tile_mutex);
    auto it = g_tile_cache.find(key);
    if (it != g_tile_cache.end()) {
      ctx->pvar = it->second.first;
      return retile(ctx, it->second.second);
    }
  }
  rapdb_status s = autotune(ctx);
  if (s != RAPDB_OK) return s;
  std::lock_guard<std::mutex> lk(g_tile_mutex);
  g_tile_cache[key] = {ctx->pvar, ctx->hi[0].I.rb};
  return RAPDB_OK;
}

// End of a stand-alone call (pass, residual, timing): wait for the stream,
// then turn an error a kernel recorded into a status, and clear it.
rapdb_status finish_standalone(rapdb_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  int err = 0;
  CK(cudaMemcpy(&err, &ctx->d_ctrl->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CK(cudaMemset(&ctx->d_ctrl->err, 0, sizeof(int)));
    return fail(ctx, RAPDB_ERR_CUDA, ctrl_error_text(err));
  }
  return RAPDB_OK;
}

// Batched contexts: one tile variant for every instance's pass (the pass
// kernel is launched once over all instances' blocks) and rows per block per
// size class.  The instances are grouped by ceil(log2 n); for each class its
// largest instance (M n^2) times every (variant, rows per block) on the pass
// its trials run (the incremental compensated pass with refinement, else the
// plain pass), CUDA events on the context's stream.  The variant with the
// least time summed over the classes, weighted by their instance counts, is
// kept, and each class takes its fastest rows per block for it.  The blocks
// were sized for the smallest tile (32 rows).
rapdb_status autotune_batched(rapdb_ctx* ctx) {
  NvtxScope nvtx_scope("rapdb_autotune_batched");
  cudaStream_t st = ctx->stream;
  const int rbs[3] = {32, 64, 128};
  std::map<int, std::vector<int>> cls;
  for (int b = 0; b < ctx->B; ++b) {
    int key = 0;
    while ((1 << key) < ctx->hi[b].I.n) ++key;
    cls[key].push_back(b);
  }
  std::vector<std::pair<int, int>> reps;            // (class key, representative instance)
  for (auto& kv : cls) {
    int best = kv.second[0];
    for (int b : kv.second) {
      const Inst& I = ctx->hi[b].I;
      const Inst& J = ctx->hi[best].I;
      if ((int64_t)I.M * I.n * I.n > (int64_t)J.M * J.n * J.n) best = b;
    }
    reps.push_back({kv.first, best});
  }
  const int nc = (int)reps.size();
  std::vector<float> t((size_t)nc * NVAR * 3, 1e30f);
  for (int c = 0; c < nc; ++c) {
    const int b = reps[c].second;
    Inst& I = ctx->hi[b].I;
    const int rb0 = I.rb;
    for (int ri = 0; ri < 3; ++ri) {
      if (ri > 0 && rbs[ri] > 2 * I.n) break;
      I.rb = rbs[ri];
      I.nrb = (I.n + I.rb - 1) / I.rb;
      CK(cudaMemcpyAsync(ctx->d_inst + b, &I, sizeof(Inst), cudaMemcpyHostToDevice, st));
      const int grid = I.M * I.nrb;
      const bool inc = I.P.refine && I.Ulo[0] != nullptr;
      const int reps_n = 5;
      for (int vi = 0; vi < NVAR; ++vi) {
        auto go = [&]() {
          if (inc)
            launch_plain(RAPDB_F32, vi, dim3(grid), st, ctx->d_inst + b, I.xf[0], I.dv, nullptr, nullptr, I.U[0],
                         ctx->tU, ctx->tW, ctx->tpart, 3, &ctx->d_ctrl->err, I.xl[0], ctx->tUo);
          else
            launch_plain(RAPDB_F32, vi, dim3(grid), st, ctx->d_inst + b, I.xf[0], I.dv, nullptr, nullptr, nullptr,
                         ctx->tU, ctx->tW, ctx->tpart, 0, &ctx->d_ctrl->err);
        };
        go();
        CK(cudaGetLastError());
        CK(cudaEventRecord(ctx->t0, st));
        for (int r = 0; r < reps_n; ++r) go();
        CK(cudaEventRecord(ctx->t1, st));
        CK(cudaEventSynchronize(ctx->t1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
        t[((size_t)c * NVAR + vi) * 3 + ri] = ms / reps_n;
      }
    }
    I.rb = rb0;
    I.nrb = (I.n + I.rb - 1) / I.rb;
  }
  {
    rapdb_status fs = finish_standalone(ctx);
    if (fs != RAPDB_OK) return fs;
  }
  int best_v = 0;
  double best_sum = 1e300;
  for (int vi = 0; vi < NVAR; ++vi) {
    double sum = 0.0;
    for (int c = 0; c < nc; ++c) {
      float tmin = 1e30f;
      for (int ri = 0; ri < 3; ++ri) tmin = std::min(tmin, t[((size_t)c * NVAR + vi) * 3 + ri]);
      sum += (double)tmin * (double)cls[reps[c].first].size();
    }
    if (sum < best_sum) {
      best_sum = sum;
      best_v = vi;
    }
  }
  ctx->pvar = best_v;
  for (int c = 0; c < nc; ++c) {
    int best_ri = 0;
    for (int ri = 1; ri < 3; ++ri)
      if (t[((size_t)c * NVAR + best_v) * 3 + ri] < t[((size_t)c * NVAR + best_v) * 3 + best_ri]) best_ri = ri;
    for (int b : cls[reps[c].first]) {
      Inst& I = ctx->hi[b].I;
      I.rb = rbs[best_ri];
      I.nrb = (I.n + I.rb - 1) / I.rb;
    }
  }
  // block maps and the instance table over the tuned tiles (builds the graph)
  return set_block_maps(ctx, std::vector<char>(ctx->B, 1));
}


static_assert(kVarRPW[SYM_ROW_VARIANT<RAPDB_F32>] == SYM_ROW_RPW<RAPDB_F32> &&
                  kVarUNR[SYM_ROW_VARIANT<RAPDB_F32>] == SYM_ROW_UNR<RAPDB_F32> &&
                  kVarRPW[SYM_ROW_VARIANT<RAPDB_FP8>] == SYM_ROW_RPW<RAPDB_FP8> &&
                  kVarUNR[SYM_ROW_VARIANT<RAPDB_FP8>] == SYM_ROW_UNR<RAPDB_FP8> &&
                  kVarNST[SYM_ROW_VARIANT<RAPDB_F32>] == 0 && kVarNST[SYM_ROW_VARIANT<RAPDB_FP8>] == 0,
              "the packed context's row-streaming tile is a register variant of the table");

// pack_sym contexts: the tile of SYM_ROW_VARIANT for the row-streaming
// passes, one resident wave of CTAs for their kernel, and one CTA per SM (at
// most one per tile) for the packed tile kernels, with their shared-memory
// stages.
rapdb_status setup_sym(rapdb_ctx* ctx) {
  const Inst& I = ctx->hi[0].I;
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int smb = (int)sym_smem_bytes();
  CK(cudaFuncSetAttribute(k_sym_tiles<RAPDB_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  CK(cudaFuncSetAttribute(k_sym_tiles<RAPDB_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  CK(cudaFuncSetAttribute(k_sym_tiles<RAPDB_FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  CK(cudaFuncSetAttribute(k_sym_plain<RAPDB_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  CK(cudaFuncSetAttribute(k_sym_plain<RAPDB_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  CK(cudaFuncSetAttribute(k_sym_plain<RAPDB_FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  int occ_tiles = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_tiles, k_sym_tiles<RAPDB_F32>, NTS, sym_smem_bytes()));
  if (occ_tiles < 1) return fail(ctx, RAPDB_ERR_CUDA, "the packed tile kernel does not fit on an SM");
  const int64_t tiles = (int64_t)I.M * I.ntile;
  const int64_t items = (int64_t)I.M * I.nrb;
  ctx->pvar = (ctx->storage == RAPDB_FP8) ? SYM_ROW_VARIANT<RAPDB_FP8> : SYM_ROW_VARIANT<RAPDB_F32>;
  ctx->sym_grid = (int)std::max<int64_t>(
      1, std::min(items, (int64_t)std::max(nsm, 1) * pass_sym_occupancy(ctx->storage)));
  ctx->sym_tile_grid = (int)std::max<int64_t>(1, std::min(tiles, (int64_t)std::max(nsm, 1) * occ_tiles));
  return RAPDB_OK;
}

int64_t body_cap(const rapdb_params& p) {
  // every trial is one body; iterations <= max_iter, trials <= max_trials each,
  // plus set-up, restart and KKT bodies
  return (int64_t)(p.max_iter + 2) * (int64_t)(p.max_trials + 2) + 1024;
}

}  // namespace

extern "C" {

void rapdb_default_params(rapdb_params* p, int32_t variant) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->variant = variant == RAPDB_XY ? RAPDB_XY : RAPDB_YX;
  p->c_nm = 1;
  p->backtracking = 1;
  p->restart = RAPDB_RESTART_FIXED;
  p->mu = 0.0;
  p->eta = 0.7;
  if (p->variant == RAPDB_YX) {
    p->c_alpha = 0.4;
    p->c_beta = 0.0;
    p->delta = 0.5;
    p->gap_first = 50;
  } else {
    p->c_alpha = 0.25;
    p->c_beta = 0.3;
    p->delta = 0.4;
    p->gap_first = 100;
  }
  p->tau_bar = 1.0;
  p->gamma0 = 1.0;
  p->restart_period = 200;
  p->restart_from_average = 0;
  p->xi = 0.04;
  p->q = 0.5;
  p->gap_every = 500;
  p->storage = RAPDB_F32;
  p->refine = 1;
  p->stall_ratio = 0.5;
  p->max_iter = 50000;
  p->max_trials = 60;
  p->kkt_every = 1;
  p->use_graph = 1;
  p->tol = 1e-6;
  p->time_limit_s = 0.0;
  p->rows_per_block = 0;
  p->gap_inner_max = 200;
  p->pass_variant = 0;
  p->dual_set = RAPDB_DUAL_NONNEG;
  p->dual_radius = 1.0;
  p->restart_warm_tau = 0;
  p->pack_sym = 0;
}

rapdb_status rapdb_create(rapdb_ctx** out, int64_t n, int64_t m, int32_t q0_kind, const float* Q,
                          const float* q0diag, const float* c, const float* d, const float* lb, const float* ub,
                          const rapdb_params* p, void* stream) {
  return rapdb_create_eq(out, n, m, q0_kind, Q, q0diag, c, d, lb, ub, 0, nullptr, nullptr, p, stream);
}

rapdb_status rapdb_create_eq(rapdb_ctx** out, int64_t n, int64_t m, int32_t q0_kind, const float* Q,
                             const float* q0diag, const float* c, const float* d, const float* lb, const float* ub,
                             int64_t p_eq, const float* A_eq, const float* b_eq, const rapdb_params* p,
                             void* stream) {
  rapdb_extras ex{};
  ex.p_eq = p_eq;
  ex.A_eq = A_eq;
  ex.b_eq = b_eq;
  return rapdb_create_ex(out, n, m, q0_kind, Q, q0diag, c, d, lb, ub, &ex, p, stream);
}

rapdb_status rapdb_create_ex(rapdb_ctx** out, int64_t n, int64_t m, int32_t q0_kind, const float* Q,
                             const float* q0diag, const float* c, const float* d, const float* lb, const float* ub,
                             const rapdb_extras* ex, const rapdb_params* p, void* stream) {
  NvtxScope nvtx_scope("rapdb_create");
  const int64_t p_eq = ex ? ex->p_eq : 0;
  const float* A_eq = ex ? ex->A_eq : nullptr;
  const float* b_eq = ex ? ex->b_eq : nullptr;
  const float* hyp_a = ex ? ex->x_hyp_a : nullptr;
  const double hyp_beta = ex ? ex->x_hyp_beta : 0.0;
  rapdb_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, RAPDB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n <= 0 || m < 0 || n > (1 << 28) || m > RAPDB_MAX_CONSTRAINTS)
    return fail(nullptr, RAPDB_ERR_INVALID, "bad sizes n, m");
  if (p_eq < 0 || m + p_eq > RAPDB_MAX_CONSTRAINTS || (p_eq > 0 && (!A_eq || !b_eq)))
    return fail(nullptr, RAPDB_ERR_INVALID, "bad equality block (p_eq, A_eq, b_eq)");
  if (q0_kind < RAPDB_Q0_DENSE || q0_kind > RAPDB_Q0_ZERO) return fail(nullptr, RAPDB_ERR_INVALID, "bad q0_kind");
  const int64_t M = (q0_kind == RAPDB_Q0_DENSE) ? m + 1 : m;
  if (M < 1) return fail(nullptr, RAPDB_ERR_INVALID, "m = 0 needs a dense Q_0 (nothing to stream otherwise)");
  if ((M > 0 && !Q) || !c || (m > 0 && !d) || !lb || !ub || (q0_kind == RAPDB_Q0_DIAG && !q0diag))
    return fail(nullptr, RAPDB_ERR_INVALID, "NULL data pointer");
  {
    rapdb_status s = check_params(nullptr, p);
    if (s != RAPDB_OK) return s;
  }
  ctx = new rapdb_ctx();
  ctx->p = *p;
  ctx->stream = (cudaStream_t)stream;
  ctx->storage = p->storage;
  ctx->variant = p->variant;
  ctx->B = 1;
  ctx->hi.resize(1);
  rapdb_status s = dalloc(ctx, &ctx->d_flags, 4);
  if (s == RAPDB_OK)
    s = build_instance(ctx, ctx->hi[0], n, m, q0_kind, Q, q0diag, c, d, lb, ub, p->rows_per_block, p_eq, A_eq,
                       b_eq, hyp_a, hyp_beta);
  ctx->hyp = hyp_a != nullptr;
  if (s == RAPDB_OK && p->storage == RAPDB_FP8) {
    const Inst& I = ctx->hi[0].I;
    s = dalloc(ctx, &ctx->XS, (size_t)std::max(I.M, 1) * I.ldv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->VS, (size_t)std::max(I.M, 1) * I.ldv);
  }
  if (s == RAPDB_OK) {
    const Inst& I = ctx->hi[0].I;
    s = dalloc(ctx, &ctx->tU, (size_t)(I.m + 1) * I.ldv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tW, (size_t)(I.m + 1) * I.ldv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tUo, (size_t)(I.m + 1) * I.ldv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->txv, (size_t)2 * I.ldv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tpart, (size_t)std::max(I.M, 1) * NDOT * I.nrb);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tvpart, (size_t)I.ncb * NVP);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tdots, (size_t)(I.m + 1) * NDOT);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->ty, (size_t)std::max(I.m, 1));
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tg, (size_t)std::max(I.m, 1));
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tout, 8);
  }
  if (s == RAPDB_OK) s = finalize_ctx(ctx);
  if (s == RAPDB_OK && p->pack_sym) {
    s = setup_sym(ctx);
  } else {
    if (s == RAPDB_OK && p->rows_per_block == 0) s = pick_tile(ctx);
    if (s == RAPDB_OK && p->rows_per_block > 0) ctx->pvar = p->pass_variant;
  }
  if (s == RAPDB_OK) s = build_graph(ctx, 32);
  if (s != RAPDB_OK) {
    g_last_error = ctx->err;
    rapdb_destroy(ctx);
    return s;
  }
  *out = ctx;
  return RAPDB_OK;
}

rapdb_status rapdb_create_batched(rapdb_ctx** out, int32_t B, const int64_t* n, const int64_t* m,
                                  const float* const* Q, const float* const* c, const float* const* d,
                                  const float* const* lb, const float* const* ub, const rapdb_params* p,
                                  void* stream) {
  NvtxScope nvtx_scope("rapdb_create_batched");
  if (!out) return fail(nullptr, RAPDB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (B <= 0 || !n || !m || !Q || !c || !d || !lb || !ub) return fail(nullptr, RAPDB_ERR_INVALID, "bad batch arguments");
  {
    rapdb_status s = check_params(nullptr, p);
    if (s != RAPDB_OK) return s;
  }
  if (p->storage != RAPDB_F32) return fail(nullptr, RAPDB_ERR_INVALID, "batched contexts use F32 storage");
  if (p->pack_sym) return fail(nullptr, RAPDB_ERR_INVALID, "pack_sym needs a single-instance context");
  for (int b = 0; b < B; ++b) {
    if (n[b] <= 0 || m[b] < 0 || m[b] > RAPDB_MAX_CONSTRAINTS || n[b] > (1 << 24))
      return fail(nullptr, RAPDB_ERR_INVALID, "bad sizes in batch");
    if (!Q[b] || !c[b] || !lb[b] || !ub[b] || (m[b] > 0 && !d[b]))
      return fail(nullptr, RAPDB_ERR_INVALID, "NULL pointer in batch");
  }
  rapdb_ctx* ctx = new rapdb_ctx();
  ctx->p = *p;
  ctx->stream = (cudaStream_t)stream;
  ctx->storage = RAPDB_F32;
  ctx->variant = p->variant;
  ctx->B = B;
  ctx->batched = true;
  ctx->hi.resize(B);
  rapdb_status s = dalloc(ctx, &ctx->d_flags, 4);
  // (with autotuning the blocks are sized for the smallest tile, 32 rows)
  for (int b = 0; b < B && s == RAPDB_OK; ++b)
    s = build_instance(ctx, ctx->hi[b], n[b], m[b], RAPDB_Q0_DENSE, Q[b], nullptr, c[b], d[b], lb[b], ub[b],
                       p->rows_per_block > 0 ? p->rows_per_block : 32);
  if (s == RAPDB_OK) s = finalize_ctx(ctx);
  if (s == RAPDB_OK && p->rows_per_block > 0) {
    // the tile from the parameters
    ctx->pvar = p->pass_variant;
    s = build_graph(ctx, 32);
  } else if (s == RAPDB_OK) {
    // autotuned tiles: stand-alone pass scratch for the largest instance
    size_t mv = 1, mp = 1;
    for (int b = 0; b < B; ++b) {
      const Inst& I = ctx->hi[b].I;
      mv = std::max(mv, (size_t)(I.m + 1) * I.ldv);
      mp = std::max(mp, (size_t)std::max(I.M, 1) * NDOT * I.nrb);
    }
    s = dalloc(ctx, &ctx->tU, mv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tW, mv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tUo, mv);
    if (s == RAPDB_OK) s = dalloc(ctx, &ctx->tpart, mp);
    if (s == RAPDB_OK) s = autotune_batched(ctx);
  }
  if (s != RAPDB_OK) {
    g_last_error = ctx->err;
    rapdb_destroy(ctx);
    return s;
  }
  *out = ctx;
  return RAPDB_OK;
}

static rapdb_status solve_common(rapdb_ctx* ctx, float* const* x, float* const* y, rapdb_info* info, bool resume) {
  NvtxScope nvtx_scope("rapdb_solve");
  cudaStream_t st = ctx->stream;
  const int B = ctx->B;
  ctx->launches = 0;
  if (!resume) {
    for (int b = 0; b < B; ++b) {
      const Inst& I = ctx->hi[b].I;
      if (!x[b] || (I.m > 0 && !y[b])) return fail(ctx, RAPDB_ERR_INVALID, "NULL x or y");
      CK(cudaMemsetAsync(I.xf[0], 0, (size_t)I.ldv * 4, st));
      CK(cudaMemcpyAsync(I.xf[0], x[b], (size_t)I.n * 4, cudaMemcpyDeviceToDevice, st));
      if (I.m > 0) {
        k_f2d<<<1, 256, 0, st>>>(y[b], I.yb[0], I.m);
        ctx->launches += 1;
      }
    }
    CK(cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), st));
    k_init_state<<<B, 256, 0, st>>>(ctx->d_inst, ctx->d_state, B, ctx->p.time_limit_s, ctx->d_flags);
    ctx->launches += 1;
    CK(cudaGetLastError());
    int flags[4];
    CK(cudaMemcpyAsync(flags, ctx->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flags[0] & 1) return fail(ctx, RAPDB_ERR_INVALID, "x0 outside the box");
    if (flags[0] & 2) return fail(ctx, RAPDB_ERR_INVALID, "x0 not on the hyperplane of X");
    if (flags[1] & 1) return fail(ctx, RAPDB_ERR_INVALID, "y0 has a negative (or NaN) entry");
    if (flags[1] & 2) return fail(ctx, RAPDB_ERR_INVALID, "y0 is not on the dual simplex");
  }
  if (ctx->batched && ctx->mapped != B) {
    // a previous solve dropped finished instances from the block maps
    CK(cudaStreamSynchronize(st));
    rapdb_status s = set_block_maps(ctx, std::vector<char>(B, 1));
    if (s != RAPDB_OK) return s;
  }
  Ctrl c0{};
  c0.active = B;
  CK(cudaMemcpyAsync(ctx->d_ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(ctx->t0, st));
  rapdb_status s = run_loop(ctx, body_cap(ctx->p));
  if (s != RAPDB_OK) return s;
  CK(cudaEventRecord(ctx->t1, st));
  CK(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(State) * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ctx->h_ctrl[0], ctx->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (ctx->h_ctrl[0].err) return fail(ctx, RAPDB_ERR_CUDA, ctrl_error_text(ctx->h_ctrl[0].err));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
  rapdb_status first_bad = RAPDB_OK;
  for (int b = 0; b < B; ++b) {
    const Inst& I = ctx->hi[b].I;
    const State& S = ctx->h_state[b];
    int status = S.phase == PH_DONE ? S.status : RAPDB_ERR_MAXITER;
    if (x && x[b]) {
      k_d2f<<<(I.n + 255) / 256, 256, 0, st>>>(I.xb[S.xcur], x[b], I.n);
      ctx->launches += 1;
    }
    if (y && y[b] && I.m > 0) {
      k_d2f<<<1, 256, 0, st>>>(I.yb[S.ycur], y[b], I.m);
      ctx->launches += 1;
    }
    if (info) {
      rapdb_info& o = info[b];
      o.iters = S.it;
      o.trials = S.trials_total;
      o.restarts = S.restarts;
      o.precision_switches = S.switches;
      o.switch_iter = S.switch_it;
      o.passes = S.passes;
      o.status = status;
      o.rel_kkt = S.rel_kkt;
      o.r_stat = S.r_stat;
      o.r_feas = S.r_feas;
      o.obj = S.obj;
      o.seconds = ms * 1e-3;
      o.launches = ctx->launches;
    }
    if (status != RAPDB_OK && first_bad == RAPDB_OK) first_bad = (rapdb_status)status;
  }
  CK(cudaStreamSynchronize(st));
  ctx->have_state = true;
  return first_bad;
}

rapdb_status rapdb_solve(rapdb_ctx* ctx, float* x, float* y, rapdb_info* info) {
  if (!ctx) return fail(nullptr, RAPDB_ERR_INVALID, "ctx is NULL");
  if (ctx->batched) return fail(ctx, RAPDB_ERR_INVALID, "use rapdb_solve_batched on a batched context");
  float* xs[1] = {x};
  float* ysv[1] = {y};
  return solve_common(ctx, xs, ysv, info, false);
}

rapdb_status rapdb_solve_batched(rapdb_ctx* ctx, float* const* x, float* const* y, rapdb_info* info) {
  if (!ctx || !x || !y) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  return solve_common(ctx, x, y, info, false);
}

rapdb_status rapdb_coupling_pass(rapdb_ctx* ctx, const float* x, const float* v, const float* uold, float* U,
                                 float* W, double* dots) {
  NvtxScope nvtx_scope("rapdb_coupling_pass");
  if (!ctx || ctx->batched) return fail(ctx, RAPDB_ERR_INVALID, "single-instance context required");
  if (!x || !v || !U || !W || !dots) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  const Inst& I = ctx->hi[0].I;
  cudaStream_t st = ctx->stream;
  // the caller's vectors are unpadded (n, and (m+1, n) row-major): stage them
  // into the context's padded scratch
  float* xpad = ctx->txv;
  float* vpad = ctx->txv + I.ldv;
  CK(cudaMemcpyAsync(xpad, x, (size_t)I.n * 4, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(vpad, v, (size_t)I.n * 4, cudaMemcpyDeviceToDevice, st));
  float* Ut = ctx->tU;
  float* Wt = ctx->tW;
  float* uo = nullptr;
  if (uold) {
    uo = ctx->tUo;
    CK(cudaMemcpy2DAsync(uo, (size_t)I.ldv * 4, uold, (size_t)I.n * 4, (size_t)I.n * 4, (size_t)(I.m + 1),
                         cudaMemcpyDeviceToDevice, st));
  }
  if (I.storage == RAPDB_FP8 || I.s_off)
    k_vec_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, xpad, vpad, uo, Ut, Wt, ctx->XS, ctx->VS, ctx->tvpart, 0);
  launch_plain(I.storage, ctx->pvar, dim3(I.M * I.nrb), st, ctx->d_inst, xpad, vpad, ctx->XS, ctx->VS, uo, Ut, Wt,
               ctx->tpart, 0, &ctx->d_ctrl->err);
  k_dots_final<<<1, NT, 0, st>>>(ctx->d_inst, ctx->tpart, ctx->tvpart, dots, xpad, vpad);
  CK(cudaGetLastError());
  CK(cudaMemcpy2DAsync(U, (size_t)I.n * 4, Ut, (size_t)I.ldv * 4, (size_t)I.n * 4, (size_t)(I.m + 1),
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpy2DAsync(W, (size_t)I.n * 4, Wt, (size_t)I.ldv * 4, (size_t)I.n * 4, (size_t)(I.m + 1),
                       cudaMemcpyDeviceToDevice, st));
  return finish_standalone(ctx);
}

rapdb_status rapdb_packed_pass(rapdb_ctx* ctx, const float* x, const float* v, const float* uold, float* U,
                               float* W, double* dots) {
  NvtxScope nvtx_scope("rapdb_packed_pass");
  if (!ctx || ctx->batched) return fail(ctx, RAPDB_ERR_INVALID, "single-instance context required");
  const Inst& I = ctx->hi[0].I;
  if (I.tsym == 0) return fail(ctx, RAPDB_ERR_INVALID, "the context has no packed tiles (pack_sym = 0)");
  if (!x || !v || !uold || !U || !W) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  cudaStream_t st = ctx->stream;
  const size_t rowb = (size_t)I.n * 4, ldb = (size_t)I.ldv * 4;
  float* xpad = ctx->txv;
  float* vpad = ctx->txv + I.ldv;
  CK(cudaMemcpyAsync(xpad, x, rowb, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(vpad, v, rowb, cudaMemcpyDeviceToDevice, st));
  const size_t off = (size_t)I.s_off * I.ldv;
  CK(cudaMemcpy2DAsync(ctx->tUo + off, ldb, uold, rowb, rowb, (size_t)I.M, cudaMemcpyDeviceToDevice, st));
  // quantised contexts: the quantised tiles (the form of the trials at their
  // quantised level); FP8 reads the pre-scaled right-hand sides s_s .* v
  const int quant = I.Qpq ? 1 : 0;
  const bool fp8 = quant && I.storage == RAPDB_FP8;
  if (fp8)
    k_vec_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, xpad, vpad, nullptr, ctx->tU, ctx->tW, ctx->XS, ctx->VS,
                                      ctx->tvpart, 0);
  if (quant) launch_sym_pieces(ctx->storage, st, ctx->d_inst, fp8 ? ctx->VS : vpad);
  launch_sym_plain(ctx->storage, dim3(ctx->sym_tile_grid), st, ctx->d_inst, fp8 ? ctx->VS : vpad, quant,
                   &ctx->d_ctrl->err);
  k_sym_rows_plain<0><<<I.M * I.tsym, NT, 0, st>>>(ctx->d_inst, xpad, nullptr, vpad, ctx->tUo, nullptr, ctx->tU,
                                                   nullptr, ctx->tW, I.spart, fp8 ? I.qscale : nullptr);
  if (dots) {
    k_sym_dots<<<1, NT, 0, st>>>(ctx->d_inst, I.spart, ctx->tdots);
    CK(cudaMemcpyAsync(dots, ctx->tdots + (size_t)I.s_off * NDOT, (size_t)I.M * NDOT * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaGetLastError());
  CK(cudaMemcpy2DAsync(U, rowb, ctx->tU + off, ldb, rowb, (size_t)I.M, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpy2DAsync(W, rowb, ctx->tW + off, ldb, rowb, (size_t)I.M, cudaMemcpyDeviceToDevice, st));
  return finish_standalone(ctx);
}

rapdb_status rapdb_kkt_residual(rapdb_ctx* ctx, const float* x, const float* y, double* rel_kkt, double* r_stat,
                                double* r_feas) {
  NvtxScope nvtx_scope("rapdb_kkt_residual");
  if (!ctx || ctx->batched) return fail(ctx, RAPDB_ERR_INVALID, "single-instance context required");
  const Inst& I = ctx->hi[0].I;
  if (!x || (I.m > 0 && !y)) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  cudaStream_t st = ctx->stream;
  float* xpad = ctx->txv;
  CK(cudaMemcpyAsync(xpad, x, (size_t)I.n * 4, cudaMemcpyDeviceToDevice, st));
  if (I.m > 0) k_f2d<<<1, 256, 0, st>>>(y, ctx->ty, I.m);
  // the most precise products the context has: compensated float32 products
  // (refine = 1), else float32 Q, else the stored Q
  const int level = I.Ulo[0] ? 2 : ((I.storage != RAPDB_F32 && I.Q32) ? 1 : 0);
  float* Ut = ctx->tU;
  float* Wt = ctx->tW;
  float* Ulo = level == 2 ? ctx->tUo : nullptr;
  float* xzero = ctx->txv + I.ldv;   // zero low part of the float32 x
  if (level == 2) CK(cudaMemsetAsync(xzero, 0, (size_t)I.ldv * 4, st));
  if (I.storage == RAPDB_FP8 && level == 0)
    k_vec_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, xpad, xpad, nullptr, Ut, Wt, ctx->XS, ctx->VS, ctx->tvpart, 0);
  else if (I.s_off)
    k_vec_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, xpad, xpad, nullptr, Ut, Wt, ctx->XS, ctx->VS, ctx->tvpart,
                                      level >= 1 ? 1 : 0);
  launch_plain(I.storage, ctx->pvar, dim3(I.M * I.nrb), st, ctx->d_inst, xpad, xpad, ctx->XS, ctx->VS, nullptr, Ut,
               Wt, ctx->tpart, level, &ctx->d_ctrl->err, xzero, Ulo);
  k_dots_final<<<1, NT, 0, st>>>(ctx->d_inst, ctx->tpart, ctx->tvpart, ctx->tdots, xpad, xpad);
  if (I.hyp_a && level != 2) CK(cudaMemsetAsync(xzero, 0, (size_t)I.ldv * 4, st));
  k_kkt_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, xpad, ctx->ty, Ut, Ulo, ctx->tvpart);
  k_kkt_final<<<1, NT, 0, st>>>(ctx->d_inst, ctx->tvpart, ctx->tdots, ctx->ty, ctx->tg, ctx->tout, xpad, xzero);
  CK(cudaGetLastError());
  double out[4];
  CK(cudaMemcpyAsync(out, ctx->tout, sizeof(out), cudaMemcpyDeviceToHost, st));
  {
    rapdb_status fs = finish_standalone(ctx);
    if (fs != RAPDB_OK) return fs;
  }
  if (rel_kkt) *rel_kkt = out[0];
  if (r_stat) *r_stat = out[1];
  if (r_feas) *r_feas = out[2];
  return RAPDB_OK;
}

rapdb_status rapdb_time_pass(rapdb_ctx* ctx, int32_t reps, int32_t level, double* ms_per_pass,
                             int64_t* bytes_per_pass) {
  NvtxScope nvtx_scope("rapdb_time_pass");
  if (!ctx || ctx->batched) return fail(ctx, RAPDB_ERR_INVALID, "single-instance context required");
  if (reps < 1) return fail(ctx, RAPDB_ERR_INVALID, "reps must be >= 1");
  const Inst& I = ctx->hi[0].I;
  cudaStream_t st = ctx->stream;
  int xcur = 0, cur_level = 0;
  if (ctx->have_state) {
    CK(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(State), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    xcur = ctx->h_state[0].xcur;
    cur_level = ctx->h_state[0].precision;
  }
  int lv = level < 0 ? cur_level : level;
  if (level < 0 && cur_level == 3) lv = 7;     // the quantised level's trial pass
  if (lv > 7 || (lv >= 1 && I.storage != RAPDB_F32 && !I.Q32) || (lv >= 2 && !I.Ulo[0]) ||
      (lv == 1 && I.storage == RAPDB_F32) || (lv >= 4 && I.tsym == 0) || (lv >= 6 && !I.Qpq))
    return fail(ctx, RAPDB_ERR_INVALID, "precision level not available in this context");
  const float* x = I.xf[xcur];
  const float* v = I.dv;
  const bool fp8s = I.storage == RAPDB_FP8 && (lv == 0 || lv >= 6);   // pre-scaled right-hand sides
  if (fp8s)
    k_vec_plain<<<I.ncb, NT, 0, st>>>(ctx->d_inst, x, v, nullptr, ctx->tU, ctx->tW, ctx->XS, ctx->VS, ctx->tvpart, 0);
  const int grid = I.M * I.nrb;
  // level 6 times the quantised tile kernel alone (its right-hand-side pieces
  // formed once, here); level 7 the whole pass, pieces included
  if (lv == 6) launch_sym_pieces(ctx->storage, st, ctx->d_inst, fp8s ? ctx->VS : v);
  auto launch = [&]() {
    if (lv >= 4) {
      const int quant = lv >= 6 ? 1 : 0;
      if (lv == 7) launch_sym_pieces(ctx->storage, st, ctx->d_inst, fp8s ? ctx->VS : v);
      launch_sym_plain(ctx->storage, dim3(ctx->sym_tile_grid), st, ctx->d_inst, (quant && fp8s) ? ctx->VS : v,
                       quant, &ctx->d_ctrl->err);
      if (lv == 4 || lv == 7)
        k_sym_rows_plain<0><<<I.M * I.tsym, NT, 0, st>>>(ctx->d_inst, x, I.xl[xcur], v, I.U[0], I.Ulo[0], ctx->tU,
                                                         ctx->tUo, ctx->tW, I.spart,
                                                         (quant && fp8s) ? I.qscale : nullptr);
    } else
      launch_plain(I.storage, ctx->pvar, dim3(grid), st, ctx->d_inst, x, v, ctx->XS, ctx->VS,
                   lv == 2 ? nullptr : I.U[0],
                   ctx->tU, ctx->tW, ctx->tpart, lv, &ctx->d_ctrl->err, I.xl[xcur], ctx->tUo);
  };
  launch();   // warm-up
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->t0, st));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(ctx->t1, st));
  CK(cudaGetLastError());
  CK(cudaEventSynchronize(ctx->t1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
  {
    rapdb_status fs = finish_standalone(ctx);
    if (fs != RAPDB_OK) return fs;
  }
  if (ms_per_pass) *ms_per_pass = (double)ms / reps;
  if (bytes_per_pass) {
    const int64_t eb = lv >= 1 ? 4 : (I.storage == RAPDB_F32 ? 4 : (I.storage == RAPDB_BF16 ? 2 : 1));
    int64_t b = (int64_t)I.M * I.n * I.n * eb;
    if (I.storage == RAPDB_FP8 && lv == 0) b += (int64_t)I.M * I.n * 4;
    if (lv >= 4) b = ctx->hi[0].qp_bytes;
    if (lv >= 6) b = ctx->hi[0].qpq_bytes;
    *bytes_per_pass = b;
  }
  return RAPDB_OK;
}

rapdb_status rapdb_get_solution_f64(rapdb_ctx* ctx, double* x, double* y) {
  if (!ctx || ctx->batched || !x) return fail(ctx, RAPDB_ERR_INVALID, "single-instance context and x required");
  if (!ctx->have_state) return fail(ctx, RAPDB_ERR_INVALID, "no solution yet (run rapdb_solve first)");
  const Inst& I = ctx->hi[0].I;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(State), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const State& S = ctx->h_state[0];
  CK(cudaMemcpyAsync(x, I.xb[S.xcur], (size_t)I.n * 8, cudaMemcpyDeviceToDevice, st));
  if (y && I.m > 0) CK(cudaMemcpyAsync(y, I.yb[S.ycur], (size_t)I.m * 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return RAPDB_OK;
}

rapdb_status rapdb_set_log(rapdb_ctx* ctx, int32_t capacity, double* tau_log, int32_t* trials_log, float* x_log,
                           float* y_log, double* kkt_log, double* gap_log, double* obj_log, double* infeas_log) {
  if (!ctx) return fail(nullptr, RAPDB_ERR_INVALID, "ctx is NULL");
  if (capacity < 0) return fail(ctx, RAPDB_ERR_INVALID, "capacity < 0");
  if (capacity > 0 && ctx->batched)
    return fail(ctx, RAPDB_ERR_INVALID, "logging needs a single-instance context");
  ctx->log_cap = capacity;
  ctx->tau_log = capacity ? tau_log : nullptr;
  ctx->trials_log = capacity ? trials_log : nullptr;
  ctx->x_log = capacity ? x_log : nullptr;
  ctx->y_log = capacity ? y_log : nullptr;
  ctx->kkt_log = capacity ? kkt_log : nullptr;
  ctx->gap_log = capacity ? gap_log : nullptr;
  ctx->obj_log = capacity ? obj_log : nullptr;
  ctx->infeas_log = capacity ? infeas_log : nullptr;
  return upload_params(ctx);
}

rapdb_status rapdb_get_instance_tile(const rapdb_ctx* ctx, int32_t instance, int32_t* rows_per_block,
                                     int32_t* variant) {
  if (!ctx || instance < 0 || instance >= ctx->B) return RAPDB_ERR_INVALID;
  if (rows_per_block) *rows_per_block = ctx->hi[instance].I.rb;
  if (variant) *variant = ctx->pvar;
  return RAPDB_OK;
}

rapdb_status rapdb_get_tile(const rapdb_ctx* ctx, int32_t* rows_per_block, int32_t* ctas, int32_t* rows_per_warp,
                            int32_t* chunks_in_flight) {
  if (!ctx) return RAPDB_ERR_INVALID;
  if (rows_per_block) *rows_per_block = ctx->hi[0].I.rb;
  if (ctas) *ctas = ctx->npblk;
  if (rows_per_warp) *rows_per_warp = kVarRPW[ctx->pvar];
  if (chunks_in_flight) *chunks_in_flight = kVarUNR[ctx->pvar];
  return RAPDB_OK;
}

// Checkpoint layout: magic, B, then per instance the State struct followed by
// x^k, x^{k-1} slots, y slots, U slots, g slots, gx slots, xcum, ycum.
static void state_blobs(rapdb_ctx* ctx, int b, std::vector<std::pair<void*, size_t>>& v) {
  Inst& I = ctx->hi[b].I;
  const size_t ldv = I.ldv, mm = std::max(I.m, 1), m1 = I.m + 1;
  for (int s = 0; s < 2; ++s) {
    v.push_back({I.xb[s], ldv * 8});
    v.push_back({I.xf[s], ldv * 4});
    v.push_back({I.xl[s], ldv * 4});
    if (I.Ulo[s]) v.push_back({I.Ulo[s], m1 * ldv * 4});
    v.push_back({I.yb[s], mm * 8});
    v.push_back({I.U[s], m1 * ldv * 4});
    v.push_back({I.gb[s], mm * 8});
    if (I.gx[s]) v.push_back({I.gx[s], ldv * 8});
  }
  if (I.xcum) v.push_back({I.xcum, ldv * 8});
  if (I.ycum) v.push_back({I.ycum, mm * 8});
  if (I.gz) v.push_back({I.gz, ldv * 8});
  if (I.gzf) v.push_back({I.gzf, ldv * 4});
  if (I.gwf) v.push_back({I.gwf, ldv * 4});
  if (I.gpf) v.push_back({I.gpf, ldv * 4});
}

rapdb_status rapdb_get_state(rapdb_ctx* ctx, void* buf, size_t* len) {
  if (!ctx || !len) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  size_t total = 16;
  std::vector<std::vector<std::pair<void*, size_t>>> blobs(ctx->B);
  for (int b = 0; b < ctx->B; ++b) {
    state_blobs(ctx, b, blobs[b]);
    total += sizeof(State);
    for (auto& pr : blobs[b]) total += pr.second;
  }
  if (!buf) {
    *len = total;
    return RAPDB_OK;
  }
  if (*len < total) return fail(ctx, RAPDB_ERR_INVALID, "buffer too small");
  if (!ctx->have_state) return fail(ctx, RAPDB_ERR_INVALID, "no solver state yet (run rapdb_solve first)");
  cudaStream_t st = ctx->stream;
  uint8_t* o = (uint8_t*)buf;
  const uint64_t magic = 0x5241504442434b31ull;  // "RAPDBCK1"
  memcpy(o, &magic, 8);
  const int64_t B = ctx->B;
  memcpy(o + 8, &B, 8);
  size_t off = 16;
  CK(cudaMemcpyAsync(o + off, ctx->d_state, sizeof(State) * ctx->B, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // states were copied contiguously; interleave layout = all states first
  off += sizeof(State) * ctx->B;
  for (int b = 0; b < ctx->B; ++b)
    for (auto& pr : blobs[b]) {
      CK(cudaMemcpyAsync(o + off, pr.first, pr.second, cudaMemcpyDeviceToHost, st));
      off += pr.second;
    }
  CK(cudaStreamSynchronize(st));
  *len = total;
  return RAPDB_OK;
}

rapdb_status rapdb_set_state(rapdb_ctx* ctx, const void* buf, size_t len) {
  if (!ctx || !buf) return fail(ctx, RAPDB_ERR_INVALID, "NULL argument");
  size_t need = 0;
  rapdb_status s = rapdb_get_state(ctx, nullptr, &need);
  if (s != RAPDB_OK) return s;
  if (len != need) return fail(ctx, RAPDB_ERR_INVALID, "checkpoint size does not match this context");
  const uint8_t* o = (const uint8_t*)buf;
  uint64_t magic;
  int64_t B;
  memcpy(&magic, o, 8);
  memcpy(&B, o + 8, 8);
  if (magic != 0x5241504442434b31ull || B != ctx->B) return fail(ctx, RAPDB_ERR_INVALID, "not a checkpoint of this context");
  cudaStream_t st = ctx->stream;
  size_t off = 16;
  std::vector<State> states(ctx->B);
  memcpy(states.data(), o + off, sizeof(State) * ctx->B);
  off += sizeof(State) * ctx->B;
  for (auto& S : states) {
    S.arrive_vec = 0;
    S.arrive_pass = 0;
    S.deadline_ns = 0;
  }
  CK(cudaMemcpyAsync(ctx->d_state, states.data(), sizeof(State) * ctx->B, cudaMemcpyHostToDevice, st));
  for (int b = 0; b < ctx->B; ++b) {
    std::vector<std::pair<void*, size_t>> blobs;
    state_blobs(ctx, b, blobs);
    for (auto& pr : blobs) {
      CK(cudaMemcpyAsync(pr.first, o + off, pr.second, cudaMemcpyHostToDevice, st));
      off += pr.second;
    }
  }
  CK(cudaStreamSynchronize(st));
  ctx->have_state = true;
  return RAPDB_OK;
}

rapdb_status rapdb_resume(rapdb_ctx* ctx, float* x, float* y, rapdb_info* info) {
  if (!ctx) return fail(nullptr, RAPDB_ERR_INVALID, "ctx is NULL");
  if (!ctx->have_state) return fail(ctx, RAPDB_ERR_INVALID, "no state to resume");
  // a finished state is reopened: DONE with MAXITER / TIMEOUT continues the loop
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(State) * ctx->B, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int b = 0; b < ctx->B; ++b) {
    State& S = ctx->h_state[b];
    if (S.phase == PH_DONE && (S.status == RAPDB_ERR_MAXITER || S.status == RAPDB_ERR_TIMEOUT)) {
      S.phase = PH_TRIAL;
      S.fresh = 1;
      S.status = RAPDB_OK;
    }
    S.deadline_ns = 0;
  }
  CK(cudaMemcpyAsync(ctx->d_state, ctx->h_state, sizeof(State) * ctx->B, cudaMemcpyHostToDevice, st));
  float* xs[1] = {x};
  float* ysv[1] = {y};
  return solve_common(ctx, xs, ysv, info, true);
}

const char* rapdb_last_error(const rapdb_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_last_error.c_str();
}

void rapdb_destroy(rapdb_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (void* q : ctx->owned) cudaFree(q);
  if (ctx->h_state) cudaFreeHost(ctx->h_state);
  if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->t0) cudaEventDestroy(ctx->t0);
  if (ctx->t1) cudaEventDestroy(ctx->t1);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  delete ctx;
}

}  // extern "C"
