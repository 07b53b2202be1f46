// Device side of the rAPDB solver: data layout, the fused coupling pass and
// small reduction helpers shared by the kernels in rapdb_kernels.cuh.
//
// One "body" of the device loop is two (xy: three) kernel launches:
//   k_vec   -- per column block of every active instance: the trial step
//              (yx: dual step with momentum, then the projected primal step
//              at the new dual point; xy: projected primal step with
//              momentum), the diagonal-Q_0 part of the pass, ||d||^2 and, on
//              a new iterate, the KKT residual partials.  The last CTA of an
//              instance to finish runs the "pre-control": the FP64 KKT
//              reduction and the stop tests.
//   k_pass  -- per (matrix, row block) of every active instance: one read of
//              the stored Q_i rows against two right-hand sides (x~ and
//              d = x~ - x^k), writing Q_i x~, Q_i d and per-block FP64 dot
//              products.  The last CTA of an instance runs the
//              "post-control": the deterministic FP64 reduction, the
//              backtracking test, the step-size / momentum update and the
//              restart rule.
//   k_vec   -- (xy only) second sweep: ||a||^2 and ||b||^2 of the xy test.
// "Last CTA" uses the fence + arrival-counter pattern: no CTA ever waits on
// another, so no co-residency is assumed and nothing spins.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include "rapdb.h"

namespace rapdb_dev {

constexpr int NT = 256;            // threads per CTA, all solver kernels
constexpr int NWARP = NT / 32;
constexpr int VCOL = 32;           // vector kernel: columns per CTA
constexpr int NGRP = NT / VCOL;    // ... and constraint groups per column
constexpr int NDOT = 5;            // dots per (matrix, row block)
constexpr int NVP = 12;            // vector-kernel partials per column block
static_assert(VCOL == 32, "constraint group 0 of the vector kernel is warp 0");
// dynamic shared memory of the vector kernel per constraint: y and y~ in
// float64 and as double-float pairs
constexpr int VEC_SMEM_PER_CON = 2 * 8 + 2 * 8;
// constraints (inequalities + equalities) per instance: the vector kernel's
// per-constraint shared memory stays within 200 KB
constexpr int RAPDB_MAX_CONSTRAINTS = 6400;
static_assert(RAPDB_MAX_CONSTRAINTS * VEC_SMEM_PER_CON <= 200 * 1024, "vector kernel shared memory");

// dot slots of one matrix i (pass output)
enum DSlot : int { D_XU = 0, D_VW = 1, D_VUO = 2, D_CX = 3, D_CV = 4 };

enum Phase : int {
  PH_INIT = 0,       // first pass: U = Q x^0, g(x^0)
  PH_TRIAL = 1,      // one trial of the backtracking loop
  PH_XY2 = 2,        // xy: after the pass, ||a||^2 and ||b||^2 sweep and the test
  PH_AVG = 3,        // restart from the weighted average: xbar (vector kernel) ...
  PH_AVGP = 8,       // ... then U = Q xbar (pass kernel)
  PH_KKT32 = 4,      // quantised storage: float32 pass at x^k for the true KKT
  PH_KKT32B = 5,     // ... and its residual sweep + the refinement decision
  PH_GAPP = 6,       // adaptive restart: power iterations for the x-subproblem's step
  PH_GAPF = 7,       // ... accelerated projected gradient on the x-subproblem
  PH_GAPV = 10,      // ... value of the smoothed gap and the restart decision
  PH_ANCHOR = 11,    // compensated levels: U = Q x^k re-formed by a direct compensated product
  PH_HYPN = 12,      // primal set with a hyperplane: the projection's scalar nu (one CTA) ...
  PH_HYPX = 13,      // ... then x = clamp(v - nu a) and the column work of the phase it serves
  PH_DONE = 9
};

// vector partial slots
enum VSlot : int {
  V_DD = 0,                                                // ||d||^2
  V_XU0 = 1, V_DW0 = 2, V_DU0 = 3, V_CX0 = 4, V_CD0 = 5,   // i = 0 dots when Q_0 is not stored
  V_RS = 6, V_GF = 7, V_GC = 8,                            // KKT: ||r_stat||^2, ||Q0x+c0||^2, ||sum y(Qx+c)||^2
  V_AA = 9, V_BB = 10,                                     // xy: ||a||^2, ||b||^2
  V_X2 = 11                                                // spare: ||x||^2 / gap term
};

struct DevParams {
  int variant, c_nm, backtracking, restart, restart_period, restart_from_average;
  int max_iter, max_trials, kkt_every, refine, gap_first, gap_every, gap_inner_max;
  int dual_simplex;     // 1: y on the simplex {y >= 0, sum y = dual_r}; 0: y >= 0
  int warm_tau;         // a restart starts from the last accepted tau instead of tau_bar
  double dual_r;
  double mu, c_alpha, c_beta, delta, eta, tau_bar, gamma0, tol, stall_ratio, xi, q;
  int log_cap;
  double* gap_log;      // smoothed-gap values, one per evaluation (capacity log_cap)
  double* kkt_log;
  double* tau_log;
  int* trials_log;
  float* x_log;
  float* y_log;
  double* obj_log;      // f(x^{k+1}) of each accepted iteration k
  double* infeas_log;   // mean_i max(g_i(x^{k+1}), 0) of each accepted iteration k
};

// Immutable description of one instance (device memory).
struct Inst {
  int n, m, M;          // variables, constraints (inequalities + equalities), stored matrices
  int m_ineq;           // constraints 1..m_ineq are inequalities; m_ineq+1..m are linear
                        // equalities a'x = b (no stored matrix, free multipliers)
  int ld;               // row stride (elements) of the stored Q
  int ld32;             // row stride of the float32 Q (refinement / KKT pass)
  int ldv;              // stride of (m+1, n) vector arrays (multiple of 16)
  int q0_kind, s_off;   // s_off = 0 when Q_0 is stored, 1 otherwise
  int storage;          // rapdb_storage of Q
  int rb, nrb;          // rows per block, blocks per matrix
  int ncb;              // column blocks of VCOL for the vector kernel
  int vblk0, pblk0;     // first vector block / pass item of this instance
  const void* Q;        // (M, n, ld) stored matrices
  const float* Q32;     // (M, n, ld32) float32 matrices or null
  const float* qscale;  // FP8: (M, ldv) symmetric scales s
  const float* q0diag;  // (ldv) diagonal of Q_0 when DIAG
  const float* c;       // (m+1, ldv)
  const double* dcon;   // (m)
  const float* lb;      // (ldv), may hold -inf
  const float* ub;      // (ldv), may hold +inf
  const float* hyp_a;   // (ldv) primal set X = box with {hyp_a'x = hyp_beta}; null: the box
  double hyp_beta;
  float2* hv;           // (ldv) the point to project onto X (double-float), vector kernel -> projection
  float2* hg;           // (ldv) grad_x L at x^k (double-float), for dist(0, grad + N_X(x))
  double dnorm;         // ||d||_2 of the constants
  double* xb[2];        // x^k / x~ master copies (ldv each, padding zero)
  float* xf[2];         // float32 copies of xb: the pass right-hand side
  float* xl[2];         // xb - xf as float32 (the low part for compensated passes)
  double* yb[2];        // y^k / y~ (m)
  float* U[2];          // Q x^k / Q x~  ((m+1, ldv))
  float* Ulo[2];        // low parts of U written by compensated passes (refine only)
  float* W;             // Q d           ((m+1, ldv))
  float* dv;            // d (ldv)
  double* gx[2];        // xy: grad_x Phi(x^k,y^k) / grad_x Phi(x^{k-1},y^{k-1}); gap: work
  double* gb[2];        // g(x^k) / g(x^{k-1})  (m)
  double* gnew;         // g(x~) of the current trial (m)
  double* part;         // (M, NDOT, nrb) pass partials
  unsigned int* mcount; // (M) per-matrix arrival counters of the pass
  // symmetric block packing (pack_sym): the upper block triangle of each
  // float32 Q_i in STB x STB tiles, read by the incremental trial passes
  const float* Qp;      // (M, ntile, STB, STB) tiles, zero outside n x n; null: none
  const int* tij;       // (ntile) tile coordinates I << 16 | J, I <= J, row-major
  float* sp;            // (2, M, T, T * STB) tile products: slot J of the rows of block I,
                        // one set per right-hand side
  const void* Qpq;      // (M, ntile, STB, STB) BF16 / FP8 codes of the stored matrices in the same
                        // tiles (quantised contexts with packing, core-matrix layout), read by the
                        // quantised level's trials on the tensor cores
  uint8_t* Pq;          // (1 or M, T) blocks of the right-hand side's pieces, the B operands of those
                        // tile products (BF16: one set for d; FP8: one per stored matrix, s_s .* d)
  float2* spart;        // (M, NDOT, T) row-block dot partials of the packed pass (double-float pairs)
  int tsym, ntile;      // T = ceil(n / STB) (0: no packing), T (T + 1) / 2
  double* vpart;        // (ncb, NVP) vector partials
  double* dots;         // (m+1, NDOT) reduced dots
  double* xcum;         // averaging: sum t_k x^{k+1}  (ldv)
  double* ycum;         // sum t_k y^{k+1}  (m)
  double* gz;           // smoothed gap: x-subproblem iterate z (ldv)
  float* gzf;           // ... its float32 copy (pass right-hand side)
  float* gwf;           // ... extrapolated point w (float32, pass right-hand side)
  float* gpf;           // ... power-iteration vector (float32, pass right-hand side)
  DevParams P;
};

// Mutable solver state of one instance (device memory, FP64 scalars).
struct State {
  double tau;           // current trial tau_k
  double tau_prev;      // tau_{k-1}
  double sigma_prev;    // sigma_{k-1}
  double gamma;         // gamma_k
  double gamma_prev;    // gamma_{k-1} (xy test)
  double alpha_k, beta_k;
  double sigma0, T, t_last;
  double rel_kkt, r_stat, r_feas, obj;
  double rel_q;         // last residual measured with the stored (quantised) Q
  double kkt_ref;       // true residual at the previous restart boundary
  double dd;            // ||d||^2 of the current trial
  double dots0[NDOT];   // i = 0 dots when Q_0 is not stored
  double gap_ref, gap_val, gap_L, gap_mu, gap_pnorm, gap_prev, gap_beta, gap_ypart;
  long long deadline_ns;
  int k, it, trial, trials_total, passes, restarts, switches;
  int phase, status, fresh, restart_note, avg_pending;
  int xcur, ycur, ucur, gcur, gxcur;
  int precision;        // 0: stored Q, 1: float32 Q, 2: float32 Q, compensated products,
                        // 3: compensated products whose trial increments Q~ d come from the
                        //    quantised packed tiles (anchored by float32 compensated products)
  int switch_it;        // iteration of the first precision switch (-1: none)
  int stall_count;      // quantised-increment level: consecutive checks without a new lowest true residual
  int hyp_ret;          // the phase a projection onto X serves (PH_TRIAL or PH_GAPF)
  double hyp_nu;        // the last projection's nu (warm start of the next)
  double hyp_t;         // the last normal-cone multiplier t of the KKT residual (warm start)
  double gap_xval;      // smoothed gap: x-part objective at z_k, kept across the projection
  int gap_iter, gap_has_ref, gap_evals, trial_ready;
  int gap_it_done;      // iteration of the last smoothed-gap evaluation (-1: none)
  int check_level;      // precision level of the pending accurate KKT check (KKT32 / KKT32B)
  unsigned int arrive_vec, arrive_pass;
  int anchor_age;       // compensated levels: accepted iterations since U was last formed by a
                        // direct product (an anchor pass follows after ANCHOR_EVERY)
  int check_due;        // a precision check runs at the next iteration's KKT test
};

struct Ctrl {
  int active;           // instances not yet done
  int err;              // a bounded wait in a kernel gave up (never expected)
  int pad_[2];
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats (about 48 significant bits).  This GPU runs float64 at a small
// fraction of its float32 rate, so the per-row and per-column sums of the
// solver's vector work use these pairs on the float32 pipe; float64 is kept
// for the per-CTA partials and the scalar control.  The error-free
// transformations are Knuth's TwoSum and the FMA-based TwoProduct; every
// operation is an explicitly rounded intrinsic, so no contraction changes
// them.  The accumulations follow the compensated dot product of Ogita, Rump
// and Oishi (2005, Dot2): the rounding error of every addition and product is
// summed alongside and folded in once at the end.
// ---------------------------------------------------------------------------
struct dflt {
  float hi, lo;
};
// a + b = s + e exactly
__device__ __forceinline__ void two_sumf(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// a + b = s + e exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ dflt fast_two_sumf(float a, float b) {
  dflt r;
  r.hi = __fadd_rn(a, b);
  r.lo = __fsub_rn(b, __fsub_rn(r.hi, a));
  return r;
}
__device__ __forceinline__ dflt df_norm(float hi, float lo) {
  float s, e;
  two_sumf(hi, lo, s, e);
  return dflt{s, e};
}
__device__ __forceinline__ dflt df_from_double(double v) {
  const float h = (float)v;
  return dflt{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to_double(dflt a) { return (double)a.hi + (double)a.lo; }
// normalised sum of two pairs
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  float s, e;
  two_sumf(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
// Compensated accumulator: acc.hi += p exactly up to the error term that goes
// to acc.lo together with the caller's own error term pe.
__device__ __forceinline__ void df_acc(dflt& acc, float p, float pe) {
  float s, e;
  two_sumf(acc.hi, p, s, e);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}
// acc += a * b for pairs a, b (the lo * lo term is below the pair's precision)
__device__ __forceinline__ void df_acc_mul(dflt& acc, dflt a, dflt b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  df_acc(acc, p, pe);
}
// acc += a * f for a pair a and a float f
__device__ __forceinline__ void df_acc_mulf(dflt& acc, dflt a, float f) {
  const float p = __fmul_rn(a.hi, f);
  const float pe = __fmaf_rn(a.lo, f, __fmaf_rn(a.hi, f, -p));
  df_acc(acc, p, pe);
}
// Sum of len >= 1 pairs src[0..len-1] in index order (L2 loads issued eight
// at a time, so the adds do not wait on one load after another).
__device__ __forceinline__ dflt df_sum_pairs(const float2* __restrict__ src, int len) {
  // the loads of a batch of 32 are all issued before its sums (entries past
  // len read as (0, 0), which TwoSum adds exactly): one memory round trip
  // per 32 pairs instead of one per pair in a ragged tail
  float2 p0 = __ldcg(src);
  dflt t = {p0.x, p0.y};
  for (int r = 1; r < len; r += 32) {
    float2 b[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) b[u] = (r + u < len) ? __ldcg(src + r + u) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 32; ++u) t = df_add(t, dflt{b[u].x, b[u].y});
  }
  return t;
}

// Fixed-order sum over the 32 lanes (xor butterfly); every lane gets the same
// sum (df_add is symmetric in its arguments: TwoSum's error term is exact).
__device__ __forceinline__ dflt df_warp_sum(dflt a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dflt b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a = df_add(a, b);
  }
  return a;
}

// Deterministic CTA sum of K doubles per thread; result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* NWARP*K */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a warp whose lanes all hold zero skips its float64 butterfly (the sum is
  // zero either way); the control steps often have data in one or two warps
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (__any_sync(0xffffffffu, v[q] != 0.0)) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) smem[warp * K + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = 0.0;
      for (int w = 0; w < NWARP; ++w) s += smem[w * K + q];
      v[q] = s;
    }
  }
  __syncthreads();
}

// Deterministic CTA sum of K doubles per thread, result in every thread.
template <int K>
__device__ __forceinline__ void block_allsum(double (&v)[K], double* smem /* NWARP*K */) {
  block_sum<K>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) smem[q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = smem[q];
  __syncthreads();
}

// Projection of v (m entries, shared or global memory) onto the simplex
// {y >= 0, sum y = r}, in place, by all threads of the CTA.  The threshold
// theta solves sum_i max(v_i - theta, 0) = r: starting from all entries,
// theta is the mean excess (sum - r)/count of the entries above the previous
// theta; it only rises, and it is exact once no entry above the previous
// theta lies at or below the new one (Michelot's finite algorithm).
__device__ __forceinline__ void proj_simplex_block(double* v, int m, double r, double* smem /* NWARP*2 */) {
  double th = -INFINITY;
  for (int pass = 0; pass <= m; ++pass) {
    double s[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      if (v[i] > th) { s[0] += v[i]; s[1] += 1.0; }
    block_allsum<2>(s, smem);
    if (!(s[1] > 0.0)) break;
    const double tn = (s[0] - r) / s[1];
    double c[1] = {0.0};
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      if (v[i] > th && v[i] <= tn) c[0] += 1.0;
    block_allsum<1>(c, smem);
    th = tn;
    if (c[0] == 0.0) break;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = fmax(v[i] - th, 0.0);
  __syncthreads();
}

// Threshold t of dist(g, N_Delta(y)) for the simplex Delta: minimises
// sum_{y_i>0} (g_i - t)^2 + sum_{y_i=0} max(g_i - t, 0)^2.  t is the mean of
// g over the support and the off-support entries above t; starting from all
// entries the mean only rises as off-support entries at or below it leave.
// All threads of the CTA; the result is valid in every thread.
__device__ __forceinline__ double simplex_cone_t_block(const double* g, const double* y, int m,
                                                       double* smem /* NWARP*2 */) {
  double t = -INFINITY;
  for (int pass = 0; pass <= m; ++pass) {
    double s[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      if (y[i] > 0.0 || g[i] > t) { s[0] += g[i]; s[1] += 1.0; }
    block_allsum<2>(s, smem);
    if (!(s[1] > 0.0)) break;
    const double tn = s[0] / s[1];
    double c[1] = {0.0};
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      if (!(y[i] > 0.0) && g[i] > t && g[i] <= tn) c[0] += 1.0;
    block_allsum<1>(c, smem);
    t = tn;
    if (c[0] == 0.0) break;
  }
  return t;
}
// The same threshold, one thread.
__device__ __forceinline__ double simplex_cone_t_serial(const double* g, const double* y, int m) {
  double t = -INFINITY;
  for (int pass = 0; pass <= m; ++pass) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < m; ++i)
      if (y[i] > 0.0 || g[i] > t) { s0 += g[i]; s1 += 1.0; }
    if (!(s1 > 0.0)) break;
    const double tn = s0 / s1;
    int c = 0;
    for (int i = 0; i < m; ++i)
      if (!(y[i] > 0.0) && g[i] > t && g[i] <= tn) ++c;
    t = tn;
    if (c == 0) break;
  }
  return t;
}

// ---------------------------------------------------------------------------
// Primal set with one hyperplane, X = {lb <= x <= ub, a'x = beta} (the
// kernel-learning problem of Sec. 5.2 minimises over {x >= 0, b'x = 0}).
// Block-wide routines (any blockDim that is a multiple of 32) in
// double-float arithmetic; `sm` holds blockDim/32 + 2 float2 and `sb` 2
// doubles of shared memory.
// ---------------------------------------------------------------------------
// Fixed-order CTA sum of a pair and of a float; every thread gets both.
__device__ __forceinline__ void df_block_allsum(dflt& a, float& f, float2* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = df_warp_sum(a);
  f = warp_sumf(f);
  if (lane == 0) sm[warp] = make_float2(a.hi, a.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    dflt t = {sm[0].x, sm[0].y};
    for (int w = 1; w < nw; ++w) t = df_add(t, dflt{sm[w].x, sm[w].y});
    sm[nw] = make_float2(t.hi, t.lo);
  }
  __syncthreads();
  if (lane == 0) sm[warp] = make_float2(f, 0.f);
  const float2 r = sm[nw];
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = sm[0].x;
    for (int w = 1; w < nw; ++w) t += sm[w].x;
    sm[nw + 1] = make_float2(t, 0.f);
  }
  __syncthreads();
  a = dflt{r.x, r.y};
  f = sm[nw + 1].x;
  __syncthreads();
}

// x at a bound of the box, compared in double-float (x = xh + xl)
__device__ __forceinline__ bool df_at_or_below(float xh, float xl, float b) { return xh < b || (xh == b && xl <= 0.f); }
__device__ __forceinline__ bool df_at_or_above(float xh, float xl, float b) { return xh > b || (xh == b && xl >= 0.f); }

// phi(nu) = a'clamp(v - nu a, lb, ub) - beta over the CTA (v = I.hv as pairs),
// the slope -sum over the free coordinates of a_j^2, and sum |a_j x_j|.
__device__ __forceinline__ void hyp_phi(const Inst& I, dflt nu, dflt& phi, float& slope, float& mag, float2* sm) {
  dflt acc = {0.f, 0.f};
  float sl = 0.f, mg = 0.f;
  for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
    const float aj = I.hyp_a[j];
    const float2 vv = I.hv[j];
    dflt na = {0.f, 0.f};
    df_acc_mulf(na, nu, aj);
    const dflt t = df_add(dflt{vv.x, vv.y}, dflt{-na.hi, -na.lo});
    const float lo = I.lb[j], hi = I.ub[j];
    dflt x;
    if (df_at_or_below(t.hi, t.lo, lo)) x = dflt{lo, 0.f};
    else if (df_at_or_above(t.hi, t.lo, hi)) x = dflt{hi, 0.f};
    else {
      x = t;
      sl = fmaf(aj, aj, sl);
    }
    df_acc_mulf(acc, x, aj);
    mg = fmaf(fabsf(aj), fabsf(x.hi), mg);
  }
  dflt a2 = df_norm(acc.hi, acc.lo);
  df_block_allsum(a2, sl, sm);
  dflt m2 = {0.f, 0.f};
  df_block_allsum(m2, mg, sm);
  phi = df_add(a2, df_from_double(-I.hyp_beta));
  slope = -sl;
  mag = mg;
}

// The scalar nu of the projection onto X: the root of phi, continuous,
// piecewise linear and non-increasing, by Newton steps on its current piece
// safeguarded by a bracket (bisection when a step leaves it, doubling while
// one side is open), from the warm start nu0.  It stops when |phi| is below
// 1e-13 of sum |a_j x_j| + |beta| (the pair arithmetic's precision), or after
// 200 steps.  Every thread returns the same nu.
__device__ __forceinline__ double hyp_proj_nu(const Inst& I, double nu0, float2* sm, double* sb) {
  double nu = nu0, lo = -INFINITY, hi = INFINITY;
  for (int it = 0; it < 200; ++it) {
    dflt ph;
    float sl, mg;
    hyp_phi(I, df_from_double(nu), ph, sl, mg, sm);
    if (threadIdx.x == 0) {
      const double phi = df_to_double(ph);
      int done = fabs(phi) <= 1e-13 * ((double)mg + fabs(I.hyp_beta)) || !(phi == phi);
      double cand = nu;
      if (!done) {
        if (phi > 0.0) lo = nu;
        else hi = nu;
        cand = (sl < 0.f) ? nu - phi / (double)sl : NAN;
        if (!(cand > lo && cand < hi)) {
          if (isfinite(lo) && isfinite(hi)) cand = 0.5 * (lo + hi);
          else if (isfinite(lo)) cand = lo + fmax(1.0, 2.0 * fabs(lo));
          else cand = hi - fmax(1.0, 2.0 * fabs(hi));
        }
        if (cand == nu) done = 1;
      }
      sb[0] = cand;
      sb[1] = done ? 1.0 : 0.0;
    }
    __syncthreads();
    nu = sb[0];
    const bool done = sb[1] != 0.0;
    __syncthreads();
    if (done) break;
  }
  return nu;
}

// ||r_stat||^2 = min over t of sum_j rho_j(g_j + t a_j)^2 for X with the
// hyperplane: rho_j(h) = max(-h, 0) at a lower bound, max(h, 0) at an upper
// bound, |h| inside (dist(0, g + N_X(x)), N_X(x) = {t a + N_box(x)}).  The
// function of t is convex and continuously differentiable; its derivative's
// root is found by safeguarded Newton steps from the warm start t0.  g = I.hg
// (pairs), x = xh + xl.  Every thread returns the value; *t_out the t.
__device__ __forceinline__ double hyp_cone_rs2(const Inst& I, const float* __restrict__ xh,
                                               const float* __restrict__ xl, double t0, double* t_out,
                                               float2* sm, double* sb) {
  double t = t0, lo = -INFINITY, hi = INFINITY;
  float F = 0.f;
  for (int it = 0; it < 200; ++it) {
    const dflt td = df_from_double(t);
    dflt d1 = {0.f, 0.f};
    float d2 = 0.f, f = 0.f;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
      const float aj = I.hyp_a[j];
      const float2 g = I.hg[j];
      dflt ta = {0.f, 0.f};
      df_acc_mulf(ta, td, aj);
      const float h = df_add(dflt{g.x, g.y}, ta).hi;
      const bool at_lo = df_at_or_below(xh[j], xl[j], I.lb[j]);
      const bool at_hi = df_at_or_above(xh[j], xl[j], I.ub[j]);
      const bool act = !(at_lo || at_hi) || (at_lo && h < 0.f) || (at_hi && h > 0.f);
      if (act) {
        const float p = __fmul_rn(aj, h);
        df_acc(d1, p, __fmaf_rn(aj, h, -p));
        d2 = fmaf(aj, aj, d2);
        f = fmaf(h, h, f);
      }
    }
    dflt D = df_norm(d1.hi, d1.lo);
    df_block_allsum(D, d2, sm);
    dflt z = {0.f, 0.f};
    df_block_allsum(z, f, sm);
    F = f;
    if (threadIdx.x == 0) {
      const double Dv = df_to_double(D);
      int done = !(Dv != 0.0) || !(d2 > 0.f);
      double cand = t;
      if (!done) {
        if (Dv < 0.0) lo = t;
        else hi = t;
        cand = t - Dv / (double)d2;
        if (!(cand > lo && cand < hi)) {
          if (isfinite(lo) && isfinite(hi)) cand = 0.5 * (lo + hi);
          else if (isfinite(lo)) cand = lo + fmax(1.0, 2.0 * fabs(lo));
          else cand = hi - fmax(1.0, 2.0 * fabs(hi));
        }
        // stop once the step no longer moves t (the piece's minimiser)
        if (fabs(cand - t) <= 1e-12 * (1.0 + fabs(t))) done = 1;
      }
      sb[0] = done ? t : cand;
      sb[1] = done ? 1.0 : 0.0;
    }
    __syncthreads();
    t = sb[0];
    const bool done = sb[1] != 0.0;
    __syncthreads();
    if (done) break;
  }
  if (t_out) *t_out = t;
  return (double)F;
}

// Arrival on a per-instance counter after this CTA's partials are written.
// Returns true in every thread of the CTA that arrives last; that CTA then
// sees the partials of all others (fence before the arrival, fence after).
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == total - 1u);
    if (s_last) *counter = 0u;     // reset for the next launch (all others arrived)
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// Stored element loaders: 16 bytes -> E floats.
template <int ST> struct Elt;
template <> struct Elt<RAPDB_F32> {
  static constexpr int E = 4;
  static constexpr int B = 4;
  __device__ __forceinline__ static void cvt(const uint4& r, float* o) {
    o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
    o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
  }
};
template <> struct Elt<RAPDB_BF16> {
  static constexpr int E = 8;
  static constexpr int B = 2;
  __device__ __forceinline__ static void cvt(const uint4& r, float* o) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};
template <> struct Elt<RAPDB_FP8> {
  static constexpr int E = 16;
  static constexpr int B = 1;
  __device__ __forceinline__ static void cvt(const uint4& r, float* o) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xffffu), __NV_E4M3);
      __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16), __NV_E4M3);
      float2 a = __half22float2(*reinterpret_cast<__half2*>(&lo));
      float2 b = __half22float2(*reinterpret_cast<__half2*>(&hi));
      o[4 * k] = a.x; o[4 * k + 1] = a.y; o[4 * k + 2] = b.x; o[4 * k + 3] = b.y;
    }
  }
};

// ---------------------------------------------------------------------------
// The fused coupling pass over one row block of one stored matrix.
//
// For rows j in [row0, row0+rows) of matrix Qm (constraint index i):
//   u_j = (Q_i x)_j,  w_j = (Q_i v)_j    (FP32 accumulation)
// written to Uo[j], Wo[j], and the block's FP64 dots
//   x_j u_j, v_j w_j, v_j uold_j, c_j x_j, c_j v_j  summed over its rows,
// stored to out[q * ostride] (q = 0..4).
// Each warp takes rows in groups of RPW; each lane streams 16-byte vectors
// of those rows (ld.global.nc, no L1 allocation) against the matching
// 16-byte slices of x and v, UNR slices in flight per row.
// FP8: `xs`/`vs` hold s .* x and s .* v (s the symmetric scales), so that
// u_j = s_j * sum_k C_jk (s_k x_k); `scale` gives s_j.
// ---------------------------------------------------------------------------
template <int ST, int RPW, int UNR>
__device__ __forceinline__ void pass_block(const uint8_t* __restrict__ Qm, int ld, int row0, int rows,
                                           const float* __restrict__ x, const float* __restrict__ v,
                                           const float* __restrict__ xs, const float* __restrict__ vs,
                                           const float* __restrict__ scale,
                                           const float* __restrict__ uold,
                                           const float* __restrict__ crow,
                                           float* __restrict__ Uo, float* __restrict__ Wo,
                                           double* __restrict__ out, int ostride, double* smem) {
  constexpr int E = Elt<ST>::E;
  constexpr int EB = Elt<ST>::B;
  // float32 storage: each 16-byte chunk's E products are summed into a fresh
  // register, and the chunk sums are added with Kahan compensation, so the
  // rounding error of a row does not grow with the length of the lane's
  // accumulation chain.  Quantised storage keeps the plain FMA chain (its
  // storage error dominates).
  constexpr bool COMP = (ST == RAPDB_F32);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const size_t rowbytes = (size_t)ld * EB;
  const float* xa = (ST == RAPDB_FP8) ? xs : x;
  const float* va = (ST == RAPDB_FP8) ? vs : v;

  for (int r = row0 + warp * RPW; r < row0 + rows; r += NWARP * RPW) {
    const int nr = min(RPW, row0 + rows - r);
    const uint8_t* p[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) p[q] = Qm + (size_t)(r + (q < nr ? q : 0)) * rowbytes;
    float acc[RPW][2], cmp[RPW][2];
#pragma unroll
    for (int q = 0; q < RPW; ++q) { acc[q][0] = 0.f; acc[q][1] = 0.f; cmp[q][0] = 0.f; cmp[q][1] = 0.f; }

    auto consume = [&](const uint4 (&raw)[RPW], const float (&xv)[E], const float (&vv)[E]) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        float qe[E];
        Elt<ST>::cvt(raw[q], qe);
        if (COMP) {
          float px = qe[0] * xv[0], pv = qe[0] * vv[0];
#pragma unroll
          for (int e = 1; e < E; ++e) {
            px = fmaf(qe[e], xv[e], px);
            pv = fmaf(qe[e], vv[e], pv);
          }
          const float yx = px - cmp[q][0];
          const float tx = acc[q][0] + yx;
          cmp[q][0] = (tx - acc[q][0]) - yx;
          acc[q][0] = tx;
          const float yv = pv - cmp[q][1];
          const float tv = acc[q][1] + yv;
          cmp[q][1] = (tv - acc[q][1]) - yv;
          acc[q][1] = tv;
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            acc[q][0] = fmaf(qe[e], xv[e], acc[q][0]);
            acc[q][1] = fmaf(qe[e], vv[e], acc[q][1]);
          }
        }
      }
    };
    auto load_rhs = [&](int cc, float (&xv)[E], float (&vv)[E]) {
#pragma unroll
      for (int e = 0; e < E; e += 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(xa + cc + e));
        float4 b = __ldg(reinterpret_cast<const float4*>(va + cc + e));
        xv[e] = a.x; xv[e + 1] = a.y; xv[e + 2] = a.z; xv[e + 3] = a.w;
        vv[e] = b.x; vv[e + 1] = b.y; vv[e + 2] = b.z; vv[e + 3] = b.w;
      }
    };

    int c0 = lane * E;
    // main loop: UNR chunks per row in flight
    for (; c0 + (UNR - 1) * 32 * E < ld; c0 += UNR * 32 * E) {
      uint4 raw[UNR][RPW];
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu)
#pragma unroll
        for (int q = 0; q < RPW; ++q)
          raw[uu][q] = (q < nr) ? ld_stream16(p[q] + (size_t)(c0 + uu * 32 * E) * EB) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu) {
        float xv[E], vv[E];
        load_rhs(c0 + uu * 32 * E, xv, vv);
        consume(raw[uu], xv, vv);
      }
    }
    // tail: fewer than UNR chunks left
    for (; c0 < ld; c0 += 32 * E) {
      uint4 raw[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q)
        raw[q] = (q < nr) ? ld_stream16(p[q] + (size_t)c0 * EB) : make_uint4(0, 0, 0, 0);
      float xv[E], vv[E];
      load_rhs(c0, xv, vv);
      consume(raw, xv, vv);
    }

    // cross-lane sums (float32 trees; the compensation terms are summed
    // separately and subtracted once)
    float uu_[RPW], ww_[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      uu_[q] = warp_sumf(acc[q][0]);
      ww_[q] = warp_sumf(acc[q][1]);
      if (COMP) {
        uu_[q] -= warp_sumf(cmp[q][0]);
        ww_[q] -= warp_sumf(cmp[q][1]);
      }
    }
    // lanes 0..nr-1 finish one row each; each such lane keeps float64 sums of
    // its rows' dot products (products of two floats are exact in float64)
    if (lane < nr) {
      const int j = r + lane;
      float u = uu_[0], w = ww_[0];
#pragma unroll
      for (int q = 1; q < RPW; ++q)
        if (lane == q) { u = uu_[q]; w = ww_[q]; }
      if (ST == RAPDB_FP8) {
        const float sj = scale[j];
        u *= sj;
        w *= sj;
      }
      Uo[j] = u;
      Wo[j] = w;
      const double xj = x[j], vj = v[j], cj = crow[j];
      dsum[0] = fma(xj, (double)u, dsum[0]);
      dsum[1] = fma(vj, (double)w, dsum[1]);
      if (uold) dsum[2] = fma(vj, (double)uold[j], dsum[2]);
      dsum[3] = fma(cj, xj, dsum[3]);
      dsum[4] = fma(cj, vj, dsum[4]);
    }
  }
  // fixed-order sum over the lanes, then over the warps
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < RPW; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) smem[warp * NDOT + q] = dsum[q];
  }
  __syncthreads();
  if (threadIdx.x < NDOT) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += smem[w * NDOT + threadIdx.x];
    out[threadIdx.x * ostride] = s;
  }
  __syncthreads();
}


// ---------------------------------------------------------------------------
// Bulk-copy staging (TMA unit): 1-D cp.async.bulk global -> shared with
// mbarrier completion.  Every wait is bounded: after ~2 s of polling the wait
// gives up, sets *err and returns false (never expected on a healthy GPU).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same copy with an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s_evict_first(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                     uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  unsigned long long limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023u) == 0 && globaltimer() - t0 > limit_ns) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The fused coupling pass with the Q rows staged through shared memory.
// Each warp owns row groups of RPW rows of the CTA's block and streams them
// through its own ring of NSTAGE slots; a slot holds CWB bytes of each of the
// group's rows (one bulk copy per row), completed on the slot's mbarrier.
// Lane 0 keeps NSTAGE slots in flight; the lanes consume 16-byte pieces from
// shared memory against x and v as in pass_block.  Same outputs as
// pass_block.  `sbuf` = NWARP*NSTAGE*RPW*CWB bytes, `bars` = NWARP*NSTAGE.
template <int ST, int RPW, int NSTAGE, int CWB>
__device__ __forceinline__ void pass_block_tma(const uint8_t* __restrict__ Qm, int ld, int row0, int rows,
                                               const float* __restrict__ x, const float* __restrict__ v,
                                               const float* __restrict__ xs, const float* __restrict__ vs,
                                               const float* __restrict__ scale,
                                               const float* __restrict__ uold,
                                               const float* __restrict__ crow,
                                               float* __restrict__ Uo, float* __restrict__ Wo,
                                               double* __restrict__ out, int ostride, double* smem,
                                               uint8_t* sbuf, uint64_t* bars, int* err) {
  constexpr int E = Elt<ST>::E;
  constexpr int EB = Elt<ST>::B;
  constexpr bool COMP = (ST == RAPDB_F32);
  static_assert(CWB % 16 == 0, "slot width must be a multiple of 16 bytes");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* xa = (ST == RAPDB_FP8) ? xs : x;
  const float* va = (ST == RAPDB_FP8) ? vs : v;
  const uint32_t rowbytes = (uint32_t)ld * EB;
  const int nchunk = (int)((rowbytes + CWB - 1) / CWB);
  uint8_t* wbuf = sbuf + (size_t)warp * NSTAGE * RPW * CWB;
  uint64_t* wbar = bars + warp * NSTAGE;
  // this warp's row groups: r = row0 + (warp + k*NWARP)*RPW
  const int ngrp_all = (rows + RPW - 1) / RPW;
  const int ngrp = (ngrp_all > warp) ? (ngrp_all - warp + NWARP - 1) / NWARP : 0;
  const int T = ngrp * nchunk;
  if (lane == 0) {
    for (int sidx = 0; sidx < NSTAGE; ++sidx) mbar_init(&wbar[sidx], 1);
    fence_proxy_async();
  }
  __syncwarp();
  auto issue = [&](int t) {   // lane 0: item t -> slot t % NSTAGE
    const int g = t / nchunk, ch = t - g * nchunk;
    const int r = row0 + (warp + g * NWARP) * RPW;
    const int nr = min(RPW, row0 + rows - r);
    const uint32_t off = (uint32_t)ch * CWB;
    const uint32_t bytes = min((uint32_t)CWB, rowbytes - off);
    const int slot = t % NSTAGE;
    mbar_expect_tx(&wbar[slot], bytes * nr);
    for (int q = 0; q < nr; ++q)
      bulk_g2s(wbuf + ((size_t)slot * RPW + q) * CWB, Qm + (size_t)(r + q) * rowbytes + off, bytes, &wbar[slot]);
  };
  if (lane == 0)
    for (int t = 0; t < NSTAGE && t < T; ++t) issue(t);

  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  float acc[RPW][2], cmp[RPW][2];
#pragma unroll
  for (int q = 0; q < RPW; ++q) { acc[q][0] = 0.f; acc[q][1] = 0.f; cmp[q][0] = 0.f; cmp[q][1] = 0.f; }
  bool ok = true;
  int t = 0;
  for (; t < T; ++t) {
    const int slot = t % NSTAGE;
    const bool got = mbar_wait_bounded(&wbar[slot], (uint32_t)((t / NSTAGE) & 1), err);
    if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
    const int g = t / nchunk, ch = t - g * nchunk;
    const int r = row0 + (warp + g * NWARP) * RPW;
    const int nr = min(RPW, row0 + rows - r);
    const uint32_t off = (uint32_t)ch * CWB;
    const int npieces = (int)(min((uint32_t)CWB, rowbytes - off) / 16);
    const uint8_t* sb = wbuf + (size_t)slot * RPW * CWB;
    for (int pc = lane; pc < npieces; pc += 32) {
      const int col = (int)(off / EB) + pc * E;
      float xv[E], vv[E];
#pragma unroll
      for (int e = 0; e < E; e += 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(xa + col + e));
        float4 b = __ldg(reinterpret_cast<const float4*>(va + col + e));
        xv[e] = a.x; xv[e + 1] = a.y; xv[e + 2] = a.z; xv[e + 3] = a.w;
        vv[e] = b.x; vv[e + 1] = b.y; vv[e + 2] = b.z; vv[e + 3] = b.w;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q < nr) {
          const uint4 raw = *reinterpret_cast<const uint4*>(sb + (size_t)q * CWB + (size_t)pc * 16);
          float qe[E];
          Elt<ST>::cvt(raw, qe);
          if (COMP) {
            float px = qe[0] * xv[0], pv = qe[0] * vv[0];
#pragma unroll
            for (int e = 1; e < E; ++e) {
              px = fmaf(qe[e], xv[e], px);
              pv = fmaf(qe[e], vv[e], pv);
            }
            const float yx = px - cmp[q][0];
            const float tx = acc[q][0] + yx;
            cmp[q][0] = (tx - acc[q][0]) - yx;
            acc[q][0] = tx;
            const float yv = pv - cmp[q][1];
            const float tv = acc[q][1] + yv;
            cmp[q][1] = (tv - acc[q][1]) - yv;
            acc[q][1] = tv;
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              acc[q][0] = fmaf(qe[e], xv[e], acc[q][0]);
              acc[q][1] = fmaf(qe[e], vv[e], acc[q][1]);
            }
          }
        }
      }
    }
    if (ch == nchunk - 1) {
      // row group complete: cross-lane sums and the row outputs
      float uu_[RPW], ww_[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        uu_[q] = warp_sumf(acc[q][0]);
        ww_[q] = warp_sumf(acc[q][1]);
        if (COMP) {
          uu_[q] -= warp_sumf(cmp[q][0]);
          ww_[q] -= warp_sumf(cmp[q][1]);
        }
        acc[q][0] = 0.f; acc[q][1] = 0.f; cmp[q][0] = 0.f; cmp[q][1] = 0.f;
      }
      if (lane < nr) {
        const int j = r + lane;
        float u = uu_[0], w = ww_[0];
#pragma unroll
        for (int q = 1; q < RPW; ++q)
          if (lane == q) { u = uu_[q]; w = ww_[q]; }
        if (ST == RAPDB_FP8) {
          const float sj = scale[j];
          u *= sj;
          w *= sj;
        }
        Uo[j] = u;
        Wo[j] = w;
        const double xj = x[j], vj = v[j], cj = crow[j];
        dsum[0] = fma(xj, (double)u, dsum[0]);
        dsum[1] = fma(vj, (double)w, dsum[1]);
        if (uold) dsum[2] = fma(vj, (double)uold[j], dsum[2]);
        dsum[3] = fma(cj, xj, dsum[3]);
        dsum[4] = fma(cj, vj, dsum[4]);
      }
    }
    __syncwarp();
    if (lane == 0 && t + NSTAGE < T) {
      fence_proxy_async();   // the slot's generic-proxy reads are done before the async write
      issue(t + NSTAGE);
    }
  }
  if (!ok && lane == 0) {
    // drain this warp's copies still in flight (bounded) before the CTA exits
    for (int t2 = t; t2 < T && t2 < t + NSTAGE; ++t2)
      mbar_wait_bounded(&wbar[t2 % NSTAGE], (uint32_t)((t2 / NSTAGE) & 1), err);
  }
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < RPW; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) smem[warp * NDOT + q] = dsum[q];
  }
  __syncthreads();
  if (threadIdx.x < NDOT) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += smem[w * NDOT + threadIdx.x];
    out[threadIdx.x * ostride] = s;
  }
  __syncthreads();
}


// The fused coupling pass with whole rows staged through shared memory.
// The CTA's row block [row0, row0+rows) of one matrix is contiguous in HBM; it
// is streamed in stages of SR = SB / rowbytes rows (one bulk copy per stage,
// NST slots in flight).  Thread t owns the 16-byte pieces t, t+NT, ... of
// every row, so its x/v slices serve all SR rows of a stage; each stage ends
// with a fixed-order CTA reduction of the rows' partial sums (warp shuffles,
// then the 8 warps in order).  Requires rowbytes <= SB (checked by the caller).
// `dsm` = [NST mbarriers | 2 x NWARP x SRMAX x 2 floats | NST x SB slots].
constexpr int SRMAX = 8;
template <int SB, int NST>
__host__ __device__ constexpr size_t rows_smem_bytes() {
  return (size_t)128 + (size_t)2 * NWARP * SRMAX * 2 * 4 + (size_t)NST * SB;
}

template <int ST, int SB, int NST>
__device__ __forceinline__ void pass_block_rows(const uint8_t* __restrict__ Qm, int ld, int row0, int rows,
                                                const float* __restrict__ x, const float* __restrict__ v,
                                                const float* __restrict__ xs, const float* __restrict__ vs,
                                                const float* __restrict__ scale,
                                                const float* __restrict__ uold,
                                                const float* __restrict__ crow,
                                                float* __restrict__ Uo, float* __restrict__ Wo,
                                                double* __restrict__ out, int ostride, double* smem,
                                                uint8_t* dsm, int* err) {
  constexpr int E = Elt<ST>::E;
  constexpr int EB = Elt<ST>::B;
  constexpr bool COMP = (ST == RAPDB_F32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* xa = (ST == RAPDB_FP8) ? xs : x;
  const float* va = (ST == RAPDB_FP8) ? vs : v;
  const uint32_t rowbytes = (uint32_t)ld * EB;
  const int npc = (int)(rowbytes / 16);                   // pieces per row
  const int SR = min(SRMAX, max(1, (int)(SB / rowbytes)));
  const int T = (rows + SR - 1) / SR;
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm);
  float* red2 = reinterpret_cast<float*>(dsm + 128);      // [2][NWARP][SRMAX][2]
  uint8_t* sbuf = dsm + 128 + (size_t)2 * NWARP * SRMAX * 2 * 4;
  if (tid == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&full[k], 1);
    fence_proxy_async();
  }
  __syncthreads();
  auto issue = [&](int t) {   // thread 0: stage t -> slot t % NST
    const int r = row0 + t * SR;
    const int nr = min(SR, row0 + rows - r);
    const int slot = t % NST;
    mbar_expect_tx(&full[slot], (uint32_t)nr * rowbytes);
    bulk_g2s(sbuf + (size_t)slot * SB, Qm + (size_t)r * rowbytes, (uint32_t)nr * rowbytes, &full[slot]);
  };
  if (tid == 0)
    for (int t = 0; t < NST && t < T; ++t) issue(t);

  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = 0; t < T; ++t) {
    const int slot = t % NST;
    const bool got = mbar_wait_bounded(&full[slot], (uint32_t)((t / NST) & 1), err);
    if (!__syncthreads_and(got)) {
      // give up: drain the copies still in flight, then leave
      if (tid == 0)
        for (int t2 = t; t2 < T && t2 < t + NST; ++t2)
          mbar_wait_bounded(&full[t2 % NST], (uint32_t)((t2 / NST) & 1), err);
      __syncthreads();
      break;
    }
    const int r = row0 + t * SR;
    const int nr = min(SR, row0 + rows - r);
    const uint8_t* sb = sbuf + (size_t)slot * SB;
    float acc[SRMAX][2], cmp[SRMAX][2];
#pragma unroll
    for (int q = 0; q < SRMAX; ++q) { acc[q][0] = 0.f; acc[q][1] = 0.f; cmp[q][0] = 0.f; cmp[q][1] = 0.f; }
    for (int pc = tid; pc < npc; pc += NT) {
      const int col = pc * E;
      float xv[E], vv[E];
#pragma unroll
      for (int e = 0; e < E; e += 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(xa + col + e));
        float4 b = __ldg(reinterpret_cast<const float4*>(va + col + e));
        xv[e] = a.x; xv[e + 1] = a.y; xv[e + 2] = a.z; xv[e + 3] = a.w;
        vv[e] = b.x; vv[e + 1] = b.y; vv[e + 2] = b.z; vv[e + 3] = b.w;
      }
#pragma unroll
      for (int q = 0; q < SRMAX; ++q) {
        if (q < nr) {
          const uint4 raw = *reinterpret_cast<const uint4*>(sb + (size_t)q * rowbytes + (size_t)pc * 16);
          float qe[E];
          Elt<ST>::cvt(raw, qe);
          if (COMP) {
            float px = qe[0] * xv[0], pv = qe[0] * vv[0];
#pragma unroll
            for (int e = 1; e < E; ++e) {
              px = fmaf(qe[e], xv[e], px);
              pv = fmaf(qe[e], vv[e], pv);
            }
            const float yx = px - cmp[q][0];
            const float tx = acc[q][0] + yx;
            cmp[q][0] = (tx - acc[q][0]) - yx;
            acc[q][0] = tx;
            const float yv = pv - cmp[q][1];
            const float tv = acc[q][1] + yv;
            cmp[q][1] = (tv - acc[q][1]) - yv;
            acc[q][1] = tv;
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              acc[q][0] = fmaf(qe[e], xv[e], acc[q][0]);
              acc[q][1] = fmaf(qe[e], vv[e], acc[q][1]);
            }
          }
        }
      }
    }
    // warp sums of each row's partials -> red2[par][warp][q]
    float* rw = red2 + (size_t)(t & 1) * NWARP * SRMAX * 2;
#pragma unroll
    for (int q = 0; q < SRMAX; ++q) {
      if (q < nr) {
        float a0 = warp_sumf(acc[q][0]), a1 = warp_sumf(acc[q][1]);
        if (COMP) {
          a0 -= warp_sumf(cmp[q][0]);
          a1 -= warp_sumf(cmp[q][1]);
        }
        if (lane == 0) {
          rw[(warp * SRMAX + q) * 2 + 0] = a0;
          rw[(warp * SRMAX + q) * 2 + 1] = a1;
        }
      }
    }
    __syncthreads();   // the slot is consumed and the warp sums are visible
    if (tid == 0 && t + NST < T) {
      fence_proxy_async();
      issue(t + NST);
    }
    if (tid < nr) {
      const int q = tid;
      float u = 0.f, w = 0.f;
      for (int wq = 0; wq < NWARP; ++wq) {
        u += rw[(wq * SRMAX + q) * 2 + 0];
        w += rw[(wq * SRMAX + q) * 2 + 1];
      }
      const int j = r + q;
      if (ST == RAPDB_FP8) {
        const float sj = scale[j];
        u *= sj;
        w *= sj;
      }
      Uo[j] = u;
      Wo[j] = w;
      const double xj = x[j], vj = v[j], cj = crow[j];
      dsum[0] = fma(xj, (double)u, dsum[0]);
      dsum[1] = fma(vj, (double)w, dsum[1]);
      if (uold) dsum[2] = fma(vj, (double)uold[j], dsum[2]);
      dsum[3] = fma(cj, xj, dsum[3]);
      dsum[4] = fma(cj, vj, dsum[4]);
    }
  }
  // fixed-order sum of the row-finishing threads' dots (threads 0..SRMAX-1 of warp 0)
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < SRMAX; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (tid < NDOT) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NDOT; ++q)
      if (q == tid) s = dsum[q];
    out[tid * ostride] = s;
  }
  __syncthreads();
  (void)smem;
}


// Compensated coupling pass (precision level 2, float32 storage): the main
// right-hand side is given as x = xh + xl (two floats); each product q*xh is
// split exactly (TwoProduct with an FMA) and summed with TwoSum, the rounding
// errors are accumulated separately, q*xl and q*v use plain FMAs.  The row
// value Q x is formed in float64 and stored as a float pair (Uoh, Uol), so the
// products carry about twice the float32 precision.  The dots use x = xh + xl
// and uold = uoh + uol.
template <int RPW, int UNR>
__device__ __forceinline__ void pass_block_prec2(const float* __restrict__ Qf, int ld, int row0, int rows,
                                                 const float* __restrict__ xh, const float* __restrict__ xl,
                                                 const float* __restrict__ v,
                                                 const float* __restrict__ uoh, const float* __restrict__ uol,
                                                 const float* __restrict__ crow,
                                                 float* __restrict__ Uoh, float* __restrict__ Uol,
                                                 float* __restrict__ Wo, double* __restrict__ out, int ostride,
                                                 double* smem) {
  const uint8_t* Qm = reinterpret_cast<const uint8_t*>(Qf);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const size_t rowbytes = (size_t)ld * 4;
  for (int r = row0 + warp * RPW; r < row0 + rows; r += NWARP * RPW) {
    const int nr = min(RPW, row0 + rows - r);
    const uint8_t* p[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) p[q] = Qm + (size_t)(r + (q < nr ? q : 0)) * rowbytes;
    float sh[RPW], ce[RPW], al[RPW], aw[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) { sh[q] = 0.f; ce[q] = 0.f; al[q] = 0.f; aw[q] = 0.f; }
    auto consume = [&](const uint4 (&raw)[RPW], int cc) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(xh + cc));
      const float4 b = __ldg(reinterpret_cast<const float4*>(xl + cc));
      const float4 d = __ldg(reinterpret_cast<const float4*>(v + cc));
      const float xv[4] = {a.x, a.y, a.z, a.w}, lv[4] = {b.x, b.y, b.z, b.w}, dv4[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        float qe[4];
        Elt<RAPDB_F32>::cvt(raw[q], qe);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // explicit round-to-nearest operations: no FMA contraction may
          // merge the product into the following sums
          const float pr = __fmul_rn(qe[e], xv[e]);
          const float pe = fmaf(qe[e], xv[e], -pr);      // exact: q*x = pr + pe
          const float t = __fadd_rn(sh[q], pr);           // TwoSum(sh, pr)
          const float z = __fsub_rn(t, sh[q]);
          const float er = __fadd_rn(__fsub_rn(sh[q], __fsub_rn(t, z)), __fsub_rn(pr, z));
          sh[q] = t;
          ce[q] = __fadd_rn(ce[q], __fadd_rn(er, pe));
          al[q] = fmaf(qe[e], lv[e], al[q]);
          aw[q] = fmaf(qe[e], dv4[e], aw[q]);
        }
      }
    };
    int c0 = lane * 4;
    for (; c0 + (UNR - 1) * 128 < ld; c0 += UNR * 128) {
      uint4 raw[UNR][RPW];
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu)
#pragma unroll
        for (int q = 0; q < RPW; ++q)
          raw[uu][q] = (q < nr) ? ld_stream16(p[q] + (size_t)(c0 + uu * 128) * 4) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu) consume(raw[uu], c0 + uu * 128);
    }
    for (; c0 < ld; c0 += 128) {
      uint4 raw[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) raw[q] = (q < nr) ? ld_stream16(p[q] + (size_t)c0 * 4) : make_uint4(0, 0, 0, 0);
      consume(raw, c0);
    }
    double uu_[RPW], ww_[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      uu_[q] = warp_sum((double)sh[q]) + warp_sum((double)ce[q]) + warp_sum((double)al[q]);
      ww_[q] = warp_sum((double)aw[q]);
    }
    if (lane < nr) {
      const int j = r + lane;
      double u = uu_[0], w = ww_[0];
#pragma unroll
      for (int q = 1; q < RPW; ++q)
        if (lane == q) { u = uu_[q]; w = ww_[q]; }
      const float uh = (float)u;
      Uoh[j] = uh;
      Uol[j] = (float)(u - (double)uh);
      Wo[j] = (float)w;
      const double xj = (double)xh[j] + (double)xl[j], vj = v[j], cj = crow[j];
      dsum[0] = fma(xj, u, dsum[0]);
      dsum[1] = fma(vj, w, dsum[1]);
      if (uoh) dsum[2] = fma(vj, (double)uoh[j] + (double)uol[j], dsum[2]);
      dsum[3] = fma(cj, xj, dsum[3]);
      dsum[4] = fma(cj, vj, dsum[4]);
    }
  }
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < RPW; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) smem[warp * NDOT + q] = dsum[q];
  }
  __syncthreads();
  if (threadIdx.x < NDOT) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += smem[w * NDOT + threadIdx.x];
    out[threadIdx.x * ostride] = s;
  }
  __syncthreads();
}


// Incremental form of the compensated pass (precision level 2, float32
// storage), for trial points x~ = x^k + d: U' = U^k + Q d, with U^k the
// double-float products at x^k (uoh + uol) and Q d formed in float32 (one
// right-hand side).  Algebraically U' = Q x~; the float32 rounding of Q d is
// of the order of eps_32 |Q||d|, so it vanishes with the step, and after
// every ANCHOR_EVERY accepted iterations an anchor pass re-forms U at the
// accepted iterate by a direct compensated product, so that these roundings
// cannot add up.  Outputs and dots as in pass_block_prec2.
constexpr int ANCHOR_EVERY = 64;
template <int RPW, int UNR>
__device__ __forceinline__ void pass_block_incr(const float* __restrict__ Qf, int ld, int row0, int rows,
                                                const float* __restrict__ xh, const float* __restrict__ xl,
                                                const float* __restrict__ v,
                                                const float* __restrict__ uoh, const float* __restrict__ uol,
                                                const float* __restrict__ crow,
                                                float* __restrict__ Uoh, float* __restrict__ Uol,
                                                float* __restrict__ Wo, double* __restrict__ out, int ostride,
                                                double* smem) {
  const uint8_t* Qm = reinterpret_cast<const uint8_t*>(Qf);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const size_t rowbytes = (size_t)ld * 4;
  for (int r = row0 + warp * RPW; r < row0 + rows; r += NWARP * RPW) {
    const int nr = min(RPW, row0 + rows - r);
    const uint8_t* p[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) p[q] = Qm + (size_t)(r + (q < nr ? q : 0)) * rowbytes;
    float aw[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) aw[q] = 0.f;
    auto consume = [&](const uint4 (&raw)[RPW], int cc) {
      const float4 d = __ldg(reinterpret_cast<const float4*>(v + cc));
      const float dv4[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        float qe[4];
        Elt<RAPDB_F32>::cvt(raw[q], qe);
#pragma unroll
        for (int e = 0; e < 4; ++e) aw[q] = fmaf(qe[e], dv4[e], aw[q]);
      }
    };
    int c0 = lane * 4;
    for (; c0 + (UNR - 1) * 128 < ld; c0 += UNR * 128) {
      uint4 raw[UNR][RPW];
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu)
#pragma unroll
        for (int q = 0; q < RPW; ++q)
          raw[uu][q] = (q < nr) ? ld_stream16(p[q] + (size_t)(c0 + uu * 128) * 4) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu) consume(raw[uu], c0 + uu * 128);
    }
    for (; c0 < ld; c0 += 128) {
      uint4 raw[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) raw[q] = (q < nr) ? ld_stream16(p[q] + (size_t)c0 * 4) : make_uint4(0, 0, 0, 0);
      consume(raw, c0);
    }
    double ww_[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) ww_[q] = warp_sum((double)aw[q]);
    if (lane < nr) {
      const int j = r + lane;
      double w = ww_[0];
#pragma unroll
      for (int q = 1; q < RPW; ++q)
        if (lane == q) w = ww_[q];
      const double uo = (double)uoh[j] + (double)uol[j];
      const double u = uo + w;
      const float uh = (float)u;
      Uoh[j] = uh;
      Uol[j] = (float)(u - (double)uh);
      Wo[j] = (float)w;
      const double xj = (double)xh[j] + (double)xl[j], vj = v[j], cj = crow[j];
      dsum[0] = fma(xj, u, dsum[0]);
      dsum[1] = fma(vj, w, dsum[1]);
      dsum[2] = fma(vj, uo, dsum[2]);
      dsum[3] = fma(cj, xj, dsum[3]);
      dsum[4] = fma(cj, vj, dsum[4]);
    }
  }
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < RPW; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) smem[warp * NDOT + q] = dsum[q];
  }
  __syncthreads();
  if (threadIdx.x < NDOT) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += smem[w * NDOT + threadIdx.x];
    out[threadIdx.x * ostride] = s;
  }
  __syncthreads();
}


// Register streaming with explicit software pipelining: the loads of the
// next UNR chunks of the RPW rows are issued before the current chunks are
// consumed, so each lane keeps 2 x UNR x RPW 16-byte loads outstanding while
// it computes.  Same arithmetic and outputs as pass_block.
template <int ST, int RPW, int UNR>
__device__ __forceinline__ void pass_block_pipe(const uint8_t* __restrict__ Qm, int ld, int row0, int rows,
                                                const float* __restrict__ x, const float* __restrict__ v,
                                                const float* __restrict__ xs, const float* __restrict__ vs,
                                                const float* __restrict__ scale,
                                                const float* __restrict__ uold,
                                                const float* __restrict__ crow,
                                                float* __restrict__ Uo, float* __restrict__ Wo,
                                                double* __restrict__ out, int ostride, double* smem) {
  constexpr int E = Elt<ST>::E;
  constexpr int EB = Elt<ST>::B;
  constexpr bool COMP = (ST == RAPDB_F32);
  constexpr int STEP = UNR * 32 * E;          // columns covered by one batch of a warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const size_t rowbytes = (size_t)ld * EB;
  const float* xa = (ST == RAPDB_FP8) ? xs : x;
  const float* va = (ST == RAPDB_FP8) ? vs : v;
  for (int r = row0 + warp * RPW; r < row0 + rows; r += NWARP * RPW) {
    const int nr = min(RPW, row0 + rows - r);
    const uint8_t* p[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) p[q] = Qm + (size_t)(r + (q < nr ? q : 0)) * rowbytes;
    float acc[RPW][2], cmp[RPW][2];
#pragma unroll
    for (int q = 0; q < RPW; ++q) { acc[q][0] = 0.f; acc[q][1] = 0.f; cmp[q][0] = 0.f; cmp[q][1] = 0.f; }
    auto load_batch = [&](int cb, uint4 (&raw)[UNR][RPW]) {
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu) {
        const int cc = cb + lane * E + uu * 32 * E;
#pragma unroll
        for (int q = 0; q < RPW; ++q)
          raw[uu][q] = (q < nr && cc < ld) ? ld_stream16(p[q] + (size_t)cc * EB) : make_uint4(0, 0, 0, 0);
      }
    };
    auto consume_batch = [&](int cb, const uint4 (&raw)[UNR][RPW]) {
#pragma unroll
      for (int uu = 0; uu < UNR; ++uu) {
        const int cc = cb + lane * E + uu * 32 * E;
        if (cc >= ld) continue;
        float xv[E], vv[E];
#pragma unroll
        for (int e = 0; e < E; e += 4) {
          float4 a = __ldg(reinterpret_cast<const float4*>(xa + cc + e));
          float4 b = __ldg(reinterpret_cast<const float4*>(va + cc + e));
          xv[e] = a.x; xv[e + 1] = a.y; xv[e + 2] = a.z; xv[e + 3] = a.w;
          vv[e] = b.x; vv[e + 1] = b.y; vv[e + 2] = b.z; vv[e + 3] = b.w;
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          float qe[E];
          Elt<ST>::cvt(raw[uu][q], qe);
          if (COMP) {
            float px = qe[0] * xv[0], pv = qe[0] * vv[0];
#pragma unroll
            for (int e = 1; e < E; ++e) {
              px = fmaf(qe[e], xv[e], px);
              pv = fmaf(qe[e], vv[e], pv);
            }
            const float yx = px - cmp[q][0];
            const float tx = acc[q][0] + yx;
            cmp[q][0] = (tx - acc[q][0]) - yx;
            acc[q][0] = tx;
            const float yv = pv - cmp[q][1];
            const float tv = acc[q][1] + yv;
            cmp[q][1] = (tv - acc[q][1]) - yv;
            acc[q][1] = tv;
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              acc[q][0] = fmaf(qe[e], xv[e], acc[q][0]);
              acc[q][1] = fmaf(qe[e], vv[e], acc[q][1]);
            }
          }
        }
      }
    };
    uint4 ra[UNR][RPW], rb[UNR][RPW];
    int cb = 0;
    load_batch(cb, ra);
    while (true) {
      const int nb = cb + STEP;
      if (nb < ld) load_batch(nb, rb);           // next batch in flight
      consume_batch(cb, ra);
      if (nb >= ld) break;
      cb = nb;
      const int nb2 = cb + STEP;
      if (nb2 < ld) load_batch(nb2, ra);
      consume_batch(cb, rb);
      if (nb2 >= ld) break;
      cb = nb2;
    }
    float uu_[RPW], ww_[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      uu_[q] = warp_sumf(acc[q][0]);
      ww_[q] = warp_sumf(acc[q][1]);
      if (COMP) {
        uu_[q] -= warp_sumf(cmp[q][0]);
        ww_[q] -= warp_sumf(cmp[q][1]);
      }
    }
    if (lane < nr) {
      const int j = r + lane;
      float u = uu_[0], w = ww_[0];
#pragma unroll
      for (int q = 1; q < RPW; ++q)
        if (lane == q) { u = uu_[q]; w = ww_[q]; }
      if (ST == RAPDB_FP8) {
        const float sj = scale[j];
        u *= sj;
        w *= sj;
      }
      Uo[j] = u;
      Wo[j] = w;
      const double xj = x[j], vj = v[j], cj = crow[j];
      dsum[0] = fma(xj, (double)u, dsum[0]);
      dsum[1] = fma(vj, (double)w, dsum[1]);
      if (uold) dsum[2] = fma(vj, (double)uold[j], dsum[2]);
      dsum[3] = fma(cj, xj, dsum[3]);
      dsum[4] = fma(cj, vj, dsum[4]);
    }
  }
#pragma unroll
  for (int q = 0; q < NDOT; ++q) {
#pragma unroll
    for (int o = 1; o < RPW; o <<= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) smem[warp * NDOT + q] = dsum[q];
  }
  __syncthreads();
  if (threadIdx.x < NDOT) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += smem[w * NDOT + threadIdx.x];
    out[threadIdx.x * ostride] = s;
  }
  __syncthreads();
}

}  // namespace rapdb_dev
