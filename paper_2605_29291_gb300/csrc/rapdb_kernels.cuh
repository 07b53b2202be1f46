// Solver kernels of the device-resident rAPDB loop (see rapdb_device.cuh for
// the body structure).  All control decisions are taken on the device by the
// last-arriving CTA of an instance, in FP64, from partial sums reduced in a
// fixed order (bit-for-bit reproducible runs).  Per-constraint work of the
// control (g_i, the test's sums, buffer moves) is spread over the CTA's
// threads; only the scalar decisions run on thread 0.
//
// Method (arXiv 2605.29291):
//   APDB-yx trial (Sec. 3.2, eq. apdb-yx-y):
//     sigma = gamma_k tau, theta = sigma_{k-1}/sigma,
//     y~ = max(0, y^k + sigma((1+theta) g(x^k) - theta g(x^{k-1}))),
//     x~ = Pi_box(x^k - tau grad_x Phi(x^k, y~)).
//   APDB-xy trial (Algorithm 1):
//     x~ = Pi_box(x^k - tau((1+theta) grad_x Phi(x^k,y^k) - theta grad_x Phi(x^{k-1},y^{k-1}))),
//     y~ = max(0, y^k + sigma g(x~)).
//   Backtracking test E_k <= -delta D_p/tau - delta D_d/sigma (Sec. 3.2 test
//   function for yx; eq. (backtracking) for xy).  For quadratics the yx test
//   reduces exactly to
//     0.5 d'Q(y~)d - |d|^2/(2tau) + (1/(2 alpha_{k+1}))|g(x~)-g(x^k)|^2
//       - (1/sigma - theta alpha_k)|y~-y^k|^2/2,
//   with d'Q(y~)d = d'Q_0 d + sum_i y~_i d'Q_i d and
//   g_i(x~) - g_i(x^k) = d'(Q_i x^k + c_i) + 0.5 d'Q_i d, all from one pass.
//   Step rule: gamma_{k+1} = gamma_k(1 + mu tau_k),
//   tau_{k+1} = tau_k sqrt(gamma_k/gamma_{k+1} (1 + c_nm tau_k/tau_{k-1}))
//   (Algorithm 1; eq. nonmonotone-tau).
//   Restarts: Algorithm 2 (fixed frequency; last iterate as in Sec. 5.1 or the
//   weighted average), eq. (ada_restart) for the adaptive rule.
#pragma once
#include "rapdb_device.cuh"

namespace rapdb_dev {

__device__ __forceinline__ bool vec_phase(int ph) {
  return ph == PH_INIT || ph == PH_TRIAL || ph == PH_XY2 || ph == PH_AVG || ph == PH_KKT32B || ph == PH_GAPP ||
         ph == PH_GAPF || ph == PH_GAPV || ph == PH_HYPX;
}
__device__ __forceinline__ bool pass_phase(int ph) {
  return ph == PH_INIT || ph == PH_TRIAL || ph == PH_AVGP || ph == PH_KKT32 || ph == PH_GAPP || ph == PH_GAPF ||
         ph == PH_GAPV || ph == PH_ANCHOR;
}
__device__ __forceinline__ bool gap_phase(int ph) { return ph == PH_GAPP || ph == PH_GAPF || ph == PH_GAPV; }

// Range checks of the checked build (RAPDB_CHECKED): a CTA whose indices or
// launch configuration are out of range records a code in Ctrl::err (the first
// one wins) and returns before touching memory; the host loop stops at its
// next poll.  No trap and no device assert.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}
enum CheckCode : int { CHK_PASS_RANGE = 101, CHK_PASS_SMEM = 102, CHK_VEC_RANGE = 111, CHK_VEC_SMEM = 112,
                       CHK_PLAIN_RANGE = 121, CHK_SYM_RANGE = 131 };

// Power iterations per smoothed-gap evaluation (first one / warm-started).
constexpr int GAP_POWER_FIRST = 30;
constexpr int GAP_POWER_WARM = 10;

// Deterministic start vector of the power iteration: a uniform value in
// [-1, 1) from a 32-bit integer hash of the column index.
__device__ __forceinline__ float hash_unit(uint32_t j) {
  uint32_t h = j * 0x9E3779B1u + 0x7F4A7C15u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  h *= 0xC2B2AE3Du;
  h ^= h >> 16;
  return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

__device__ __forceinline__ void finish(State& S, Ctrl* ctrl, int status) {
  S.phase = PH_DONE;
  S.status = status;
  atomicSub(&ctrl->active, 1);
}

// Reset of Algorithm 1's initialisation line at a (re)start:
// tau_{-1} = tau_0 = tau_bar, sigma_{-1} = gamma_0 tau_bar, gamma = gamma_0,
// alpha_0 / beta_0 from the parameter recurrences at k = -1.  With warm_tau
// a restart (after at least one accepted iteration) starts from the last
// accepted tau instead of tau_bar.
static __device__ void restart_scalars(const DevParams& P, State& S) {
  const double t0 = (P.warm_tau && S.k > 0 && S.tau_prev > 0.0) ? S.tau_prev : P.tau_bar;
  S.tau_prev = t0;
  S.sigma_prev = P.gamma0 * t0;
  S.gamma = P.gamma0;
  S.tau = t0;
  if (P.variant == RAPDB_YX) {
    S.alpha_k = P.c_alpha / S.sigma_prev;
    S.beta_k = 0.0;
  } else {
    S.alpha_k = P.c_alpha / t0;
    S.beta_k = P.gamma0 * P.c_beta / S.sigma_prev;
  }
  S.k = 0;
  S.T = 0.0;
  S.trial = 0;
}

// Precision refinement: level 0 = the stored Q (float32, bfloat16 or FP8),
// 1 = float32 Q (from quantised storage), 2 = float32 Q with compensated
// (double-float) products, 3 = level 2 whose trial increments Q~ d come from
// the quantised packed tiles (U^k stays a compensated float32 product,
// re-anchored at each check).  At restart boundaries (levels 0, 1), every
// ANCHOR_EVERY accepted iterations (level 3), and when the current level
// reports convergence, the residual is checked at level 2; a stall (or a
// disagreement at convergence) switches to level 2.
__device__ __forceinline__ bool can_refine(const Inst& I, const State& S) {
  return I.P.refine && (S.precision < 2 || S.precision == 3) && (I.storage == RAPDB_F32 || I.Q32 != nullptr);
}
// The next level is always the compensated one: its trial products are
// incremental (U^k + Q d, one float32 right-hand side), so they cost what a
// plain float32 pass costs, and float32 products alone leave a KKT floor.
__device__ __forceinline__ int next_level(const Inst& I, const State& S) {
  (void)I;
  (void)S;
  return 2;
}
__device__ __forceinline__ void start_check(const Inst& I, State& S) {
  S.check_level = next_level(I, S);
  S.phase = PH_KKT32;
}

// Per-constraint terms of the feasibility residual: r_feas_i^2 and
// (g_i - d_i)^2, summed over this thread's constraints.
// All threads of the CTA (a simplex dual first finds the normal-cone
// threshold t: r_feas = dist(g, N_Delta(y)) with components g_i - t on the
// support of y and max(g_i - t, 0) off it).
__device__ __forceinline__ void kkt_feas_terms(const Inst& I, const double* g, const double* y, double& rf2,
                                               double& gd2, double* smem) {
  rf2 = 0.0;
  gd2 = 0.0;
  const double t = I.P.dual_simplex ? simplex_cone_t_block(g, y, I.m_ineq, smem) : 0.0;
  for (int i = threadIdx.x; i < I.m; i += NT) {
    const double gi = g[i];
    double ri;
    if (i >= I.m_ineq) ri = gi;                 // equality: |a'x - b|
    else if (I.P.dual_simplex) ri = (y[i] > 0.0) ? gi - t : fmax(gi - t, 0.0);
    else ri = (y[i] > 0.0) ? fabs(gi) : fmax(gi, 0.0);
    rf2 += ri * ri;
    const double dv = gi - I.dcon[i];
    gd2 += dv * dv;
  }
}

__device__ __forceinline__ void kkt_finish(const Inst& I, double rs2, double gf2, double gc2, double rf2,
                                           double gd2, double& rel, double& r_stat, double& r_feas) {
  r_stat = sqrt(rs2);
  r_feas = sqrt(rf2);
  const double den_s = 1.0 + fmax(sqrt(gf2), sqrt(gc2));
  const double den_f = 1.0 + fmax(I.dnorm, sqrt(gd2));
  rel = fmax(r_stat / den_s, r_feas / den_f);
}

// Acceptance, vector part (all threads of the CTA): g^{k-1} <- g^k is done by
// writing g(x~) over the old slot, and the dual average sum.  k0, gcur0,
// ycur0, t are the values read before any scalar update.
__device__ __forceinline__ void accept_vectors(const Inst& I, int k0, int gcur0, int ycur0, double t) {
  double* gdst = I.gb[gcur0 ^ 1];
  const double* yn = I.yb[ycur0 ^ 1];
  for (int i = threadIdx.x; i < I.m; i += NT) {
    gdst[i] = I.gnew[i];
    if (I.P.restart_from_average) I.ycum[i] = (k0 == 0 ? 0.0 : I.ycum[i]) + t * yn[i];
  }
}

// Acceptance, scalar part (thread 0, after accept_vectors and a barrier):
// averaging weights, step rule, buffer swaps, logging and the
// fixed-frequency restart rule.
static __device__ void accept_scalars(const Inst& I, State& S, double sigma, double alpha_next, double beta_next) {
  const DevParams& P = I.P;
  const double tau = S.tau;
  const int trials_this = S.trial + 1;
  if (S.k == 0) S.sigma0 = sigma;
  const double t = sigma / S.sigma0;
  S.T += t;
  S.t_last = t;
  double gnext = S.gamma, tnext = tau;
  if (P.backtracking) {
    gnext = S.gamma * (1.0 + P.mu * tau);
    tnext = tau * sqrt(S.gamma / gnext * (1.0 + (double)P.c_nm * tau / S.tau_prev));
  }
  if (S.it < P.log_cap) {
    if (P.tau_log) P.tau_log[S.it] = tau;
    if (P.trials_log) P.trials_log[S.it] = trials_this;
  }
  // compensated levels: the accepted products came from U^k + Q d; after
  // ANCHOR_EVERY of them an anchor pass re-forms U at the new iterate
  if (S.precision >= 2) S.anchor_age += 1;
  S.tau_prev = tau;
  S.sigma_prev = sigma;
  S.alpha_k = alpha_next;
  S.beta_k = beta_next;
  S.gamma = gnext;
  S.tau = tnext;
  S.xcur ^= 1;
  S.ycur ^= 1;
  S.ucur ^= 1;
  S.gcur ^= 1;
  S.gxcur ^= 1;
  S.k += 1;
  S.it += 1;
  S.trial = 0;
  S.fresh = 1;
  S.obj = 0.5 * __ldcg(&I.dots[D_XU]) + __ldcg(&I.dots[D_CX]);
  if (S.it - 1 < P.log_cap) {
    if (P.obj_log) P.obj_log[S.it - 1] = S.obj;
    if (P.infeas_log) {
      double v = 0.0;
      for (int i = 0; i < I.m; ++i) v += fmax(__ldcg(&I.gnew[i]), 0.0);
      P.infeas_log[S.it - 1] = I.m > 0 ? v / I.m : 0.0;
    }
  }
  S.phase = PH_TRIAL;
  // levels 0 and 1 are checked at restart boundaries and every
  // restart_period / 4 iterations; level 3 at its anchors (below)
  const bool periodic = can_refine(I, S) && S.precision < 2;
  if (P.restart == RAPDB_RESTART_FIXED && S.k == P.restart_period) {
    if (P.restart_from_average) {
      S.avg_pending = 1;
    } else {
      restart_scalars(P, S);
      S.restart_note = 1;
      if (periodic) S.check_due = 1;
    }
  } else if (periodic && P.restart_period > 0 && S.it % max(1, P.restart_period / 4) == 0) {
    S.check_due = 1;
  }
  // the anchor pass comes first (a restart from the average forms U
  // directly); at level 3 the precision check is the anchor: its direct
  // compensated pass at x^k replaces U^k unless the check ends the solve
  if (S.precision >= 2 && S.anchor_age >= ANCHOR_EVERY && !S.avg_pending) {
    if (S.precision == 3) S.check_due = 1;
    else S.phase = PH_ANCHOR;
  }
}

static __device__ void reject_trial(const Inst& I, State& S, Ctrl* ctrl) {
  S.trial += 1;
  if (S.trial >= I.P.max_trials) {
    finish(S, ctrl, RAPDB_ERR_BACKTRACK);
    return;
  }
  S.tau *= I.P.eta;
  S.phase = PH_TRIAL;
}

// ---------------------------------------------------------------------------
// k_vec: trial step / KKT partials / xy second sweep / restart points.
// A CTA covers VCOL columns; its NGRP thread groups split the constraint sum
// of each column (fixed-order combination in shared memory).
// ---------------------------------------------------------------------------
template <int ST>
__global__ void __launch_bounds__(NT) k_vec(const Inst* __restrict__ insts, State* __restrict__ states,
                                            Ctrl* __restrict__ ctrl, const int* __restrict__ vmap,
                                            float* __restrict__ XS, float* __restrict__ VS) {
  extern __shared__ double sm[];            // ys[m], yts[m] (float64), then ydf[m], ytdf[m] (double-float)
  __shared__ double red[NWARP * NVP];
  __shared__ double vfin[NVP];
  __shared__ float2 pg[3][NGRP][VCOL];      // the groups' double-float constraint sums
  __shared__ float sx[VCOL], sd[VCOL];
  __shared__ int s_dec;
  __shared__ __align__(16) State Sc;        // the control step's copy of the state
  __shared__ __align__(16) Inst sI;         // the instance descriptor (one parallel copy)
  const int b = vmap[blockIdx.x];
  {
    // the instance descriptor and the state in shared memory, in one round
    // trip: the column work below only reads the state (the last CTA copies
    // it again for the control step, and the arrival counter is global)
    const uint32_t* isrc = reinterpret_cast<const uint32_t*>(&insts[b]);
    uint32_t* idst = reinterpret_cast<uint32_t*>(&sI);
    for (int w = threadIdx.x; w < (int)(sizeof(Inst) / 4); w += NT) idst[w] = isrc[w];
    const uint32_t* ssrc = reinterpret_cast<const uint32_t*>(&states[b]);
    uint32_t* sdst = reinterpret_cast<uint32_t*>(&Sc);
    for (int w = threadIdx.x; w < (int)(sizeof(State) / 4); w += NT) sdst[w] = ssrc[w];
  }
  __syncthreads();
  const State& S = Sc;
  const int phase = S.phase;
  if (!vec_phase(phase)) return;
  const Inst& I = sI;
  const DevParams& P = I.P;
  const int m = I.m, n = I.n, ldv = I.ldv;
  const int cb = blockIdx.x - I.vblk0;
  const int tid = threadIdx.x;
#ifdef RAPDB_CHECKED
  {
    const int code = !(cb >= 0 && cb < I.ncb) ? CHK_VEC_RANGE
                     : (dyn_smem_bytes() < (unsigned)m * (unsigned)VEC_SMEM_PER_CON ? CHK_VEC_SMEM : 0);
    if (code) {
      if (tid == 0) atomicCAS(&ctrl->err, 0, code);
      return;
    }
  }
#endif
  const int lc = tid % VCOL, grp = tid / VCOL;
  const int fresh = S.fresh;
  const int k = S.k, it = S.it;
  double* ys = sm;
  double* yts = sm + m;
  float2* ydf = reinterpret_cast<float2*>(sm + 2 * m);
  float2* ytdf = ydf + m;

  const double tau = S.tau;
  const double sigma = S.gamma * tau;
  const double theta = S.sigma_prev / sigma;
  const int ycur0 = S.ycur, gcur0 = S.gcur;
  const double* ycur = I.yb[ycur0];
  const double* gk = I.gb[gcur0];
  const double* gp = (k == 0) ? gk : I.gb[gcur0 ^ 1];
  for (int i = tid; i < m; i += NT) {
    ys[i] = ycur[i];
    if (phase == PH_TRIAL && P.variant == RAPDB_YX) {
      const double s = (1.0 + theta) * gk[i] - theta * gp[i];
      // inequality multipliers: max(0, .) or the simplex below; equality multipliers are free
      yts[i] = (P.dual_simplex || i >= I.m_ineq) ? ycur[i] + sigma * s : fmax(0.0, ycur[i] + sigma * s);
    } else if (phase == PH_XY2) {
      yts[i] = I.yb[ycur0 ^ 1][i];
    } else {
      yts[i] = ycur[i];
    }
  }
  __syncthreads();
  if (P.dual_simplex && phase == PH_TRIAL && P.variant == RAPDB_YX) proj_simplex_block(yts, I.m_ineq, P.dual_r, red);
  if (cb == 0 && phase == PH_TRIAL && P.variant == RAPDB_YX)
    for (int i = tid; i < m; i += NT) I.yb[ycur0 ^ 1][i] = yts[i];
  // double-float copies of the multipliers for the column sums (XY2: of y~ - y)
  for (int i = tid; i < m; i += NT) {
    const dflt a = df_from_double(ys[i]);
    const dflt b = df_from_double(phase == PH_XY2 ? yts[i] - ys[i] : yts[i]);
    ydf[i] = make_float2(a.hi, a.lo);
    ytdf[i] = make_float2(b.hi, b.lo);
  }
  __syncthreads();

  const bool kkt_due = (phase == PH_TRIAL && fresh &&
                        ((P.kkt_every > 0 && it % P.kkt_every == 0) || it >= P.max_iter)) ||
                       phase == PH_KKT32B;
  // adaptive restart: a smoothed-gap evaluation is due before this iteration
  const bool gap_due = phase == PH_TRIAL && fresh && P.restart == RAPDB_RESTART_GAP && it >= P.gap_first &&
                       (it == P.gap_first || (it - P.gap_first) % P.gap_every == 0) && S.gap_it_done != it;
  const int gap_iter = S.gap_iter;
  const int gap_P = (S.gap_evals == 0) ? GAP_POWER_FIRST : GAP_POWER_WARM;
  const double* xk = I.xb[S.xcur];
  double* xt_out = I.xb[S.xcur ^ 1];
  float* xt_out32 = I.xf[S.xcur ^ 1];
  float* xt_outlo = I.xl[S.xcur ^ 1];
  const float* Uc = I.U[S.ucur];
  float* Un = I.U[S.ucur ^ 1];
  // low parts of U when the products were formed with compensation
  const bool comp_lv = S.precision >= 2;
  const float* Uclo = comp_lv ? I.Ulo[S.ucur] : nullptr;
  const float* Unlo = (phase == PH_KKT32B ? S.check_level == 2 : (comp_lv && phase == PH_XY2))
                          ? I.Ulo[S.ucur ^ 1] : nullptr;
  const float* c = I.c;
  double acc[NVP];
#pragma unroll
  for (int q = 0; q < NVP; ++q) acc[q] = 0.0;

  const int j = cb * VCOL + lc;
  // ---- constraint sums, split over the NGRP groups ----
  // Compensated double-float accumulation: each term y_i * (U_ij + Ulo_ij +
  // c_ij) is a TwoProduct of pairs, its rounding errors summed alongside.
  {
    dflt s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f};
    if (j < n) {
      if (phase == PH_TRIAL || phase == PH_KKT32B || phase == PH_XY2) {
        // TRIAL / KKT32B: sum y_i (u_i + c_i) and sum y~_i (u_i + c_i);
        // XY2: sum (y~_i - y_i)(u~_i + c_i) and sum y_i w_i
        const bool xy2 = phase == PH_XY2;
        const float* Us = (phase == PH_TRIAL) ? Uc : Un;
        const float* Ul = (phase == PH_TRIAL) ? Uclo : Unlo;
        for (int i = 1 + grp; i <= m; i += NGRP) {
          const size_t o = (size_t)i * ldv + j;
          float vh, ve;
          two_sumf(Us[o], c[o], vh, ve);
          const dflt v = {vh, __fadd_rn(ve, Ul ? Ul[o] : 0.f)};
          const float2 a = ydf[i - 1], b = ytdf[i - 1];
          if (xy2) {
            df_acc_mul(s0, dflt{b.x, b.y}, v);
            df_acc_mulf(s1, dflt{a.x, a.y}, I.W[o]);
          } else {
            df_acc_mul(s0, dflt{a.x, a.y}, v);
            df_acc_mul(s1, dflt{b.x, b.y}, v);
          }
        }
      } else if (gap_phase(phase)) {
        // sum_i y_i (Q_i w)_j, sum_i y_i (Q_i z)_j, sum_i y_i c_ij
        for (int i = 1 + grp; i <= m; i += NGRP) {
          const size_t o = (size_t)i * ldv + j;
          const float2 a = ydf[i - 1];
          df_acc_mulf(s0, dflt{a.x, a.y}, Un[o]);
          df_acc_mulf(s1, dflt{a.x, a.y}, I.W[o]);
          df_acc_mulf(s2, dflt{a.x, a.y}, c[o]);
        }
      }
    }
    pg[0][grp][lc] = make_float2(s0.hi, s0.lo);
    pg[1][grp][lc] = make_float2(s1.hi, s1.lo);
    pg[2][grp][lc] = make_float2(s2.hi, s2.lo);
  }
  __syncthreads();

  if (grp == 0 && j < n) {
    double gc, gt, g2;
    {
      dflt a = df_norm(pg[0][0][lc].x, pg[0][0][lc].y), b = df_norm(pg[1][0][lc].x, pg[1][0][lc].y),
           e = df_norm(pg[2][0][lc].x, pg[2][0][lc].y);
#pragma unroll
      for (int g = 1; g < NGRP; ++g) {
        a = df_add(a, dflt{pg[0][g][lc].x, pg[0][g][lc].y});
        b = df_add(b, dflt{pg[1][g][lc].x, pg[1][g][lc].y});
        e = df_add(e, dflt{pg[2][g][lc].x, pg[2][g][lc].y});
      }
      gc = df_to_double(a);
      gt = df_to_double(b);
      g2 = df_to_double(e);
    }
    const double xj = xk[j];
    const float xj32 = I.xf[S.xcur][j];
    const double c0 = c[j];
    const double q0d = (I.q0_kind == RAPDB_Q0_DIAG) ? (double)I.q0diag[j] : 0.0;
    // The trial point x~ and its column work (the pass's right-hand sides,
    // ||d||^2, the diagonal Q_0 row and the i = 0 dots).  u0 = (Q_0 x^k)_j.
    auto trial_final = [&](double xt, double u0) {
      // the iterate is kept in float64 (steps far below one float32 ulp of
      // x still move it); the pass reads float32 copies of x~ and of d
      const float xt32 = (float)xt;
      const float d32 = (float)(xt - xj);
      xt_out[j] = xt;
      xt_out32[j] = xt32;
      xt_outlo[j] = (float)(xt - (double)xt32);
      I.dv[j] = d32;
      sx[lc] = xt32;
      sd[lc] = d32;
      acc[V_DD] = (double)d32 * (double)d32;
      if (I.s_off) {
        const double u0d = q0d * (comp_lv ? xt : (double)xt32);
        const float u0n = (float)u0d;
        const float w0 = (float)(q0d * (double)d32);
        Un[j] = u0n;
        if (comp_lv) I.Ulo[S.ucur ^ 1][j] = (float)(u0d - (double)u0n);
        I.W[j] = w0;
        acc[V_XU0] = (comp_lv ? xt : (double)xt32) * u0d;
        acc[V_DW0] = (double)d32 * (double)w0;
        acc[V_DU0] = (double)d32 * u0;
      }
      acc[V_CX0] = c0 * (double)xt32;
      acc[V_CD0] = c0 * (double)d32;
    };
    // One accelerated-gradient step of the smoothed gap's x-subproblem, from
    // z_k, w_k to z_{k+1} = zn (already projected onto X).
    auto gapf_final = [&](double zn) {
      const double zk = I.gz[j];
      const float wj = I.gwf[j];
      const double wn = zn + S.gap_beta * (zn - zk);                  // momentum of this step
      I.gz[j] = zn;
      I.gzf[j] = (float)zn;
      I.gwf[j] = (float)wn;
      sx[lc] = (float)wn;
      sd[lc] = (float)zn;
      acc[0] = (zn - zk) * (zn - zk);
      acc[1] = zn * zn;
      acc[5] = (zn - (double)wj) * (zn - (double)wj);                // |z+ - w|^2 (gradient mapping / L)
    };
    // the point to project onto X with the hyperplane, kept as a pair
    auto keep_for_projection = [&](double v) {
      const dflt vd = df_from_double(v);
      I.hv[j] = make_float2(vd.hi, vd.lo);
    };
    if (phase == PH_HYPX) {
      // projection onto X: x = clamp(v - nu a) with the nu of the projection kernel
      const float2 vv = I.hv[j];
      const dflt nu = df_from_double(S.hyp_nu);
      dflt na = {0.f, 0.f};
      df_acc_mulf(na, nu, I.hyp_a[j]);
      const dflt t = df_add(dflt{vv.x, vv.y}, dflt{-na.hi, -na.lo});
      const double xp = df_at_or_below(t.hi, t.lo, I.lb[j]) ? (double)I.lb[j]
                        : (df_at_or_above(t.hi, t.lo, I.ub[j]) ? (double)I.ub[j] : df_to_double(t));
      if (S.hyp_ret == PH_TRIAL) trial_final(xp, I.s_off ? q0d * xj : 0.0);
      else gapf_final(xp);
    } else if (phase == PH_TRIAL || phase == PH_KKT32B) {
      const float* Us = (phase == PH_KKT32B) ? Un : Uc;
      const float* Ul = (phase == PH_KKT32B) ? Unlo : Uclo;
      const double u0 = (I.s_off ? q0d * xj : (double)Us[j] + (Ul ? (double)Ul[j] : 0.0));
      const double gf = u0 + c0;
      const double grad = gf + gc;
      if (kkt_due) {
        if (I.hyp_a) {
          // dist(0, grad + N_X(x)) needs every column: the control CTA forms it
          const dflt gd = df_from_double(grad);
          I.hg[j] = make_float2(gd.hi, gd.lo);
        } else {
          const double lo = I.lb[j], hi = I.ub[j];
          const double rs = (xj <= lo) ? fmax(-grad, 0.0) : ((xj >= hi) ? fmax(grad, 0.0) : fabs(grad));
          acc[V_RS] = rs * rs;
        }
        acc[V_GF] = gf * gf;
        acc[V_GC] = gc * gc;
      }
      if (phase == PH_KKT32B) {
        if (I.s_off) {
          const double u0n = q0d * xj;
          Un[j] = (float)u0n;
          if (Unlo) I.Ulo[S.ucur ^ 1][j] = (float)(u0n - (double)(float)u0n);
        }
      } else {
        double step;
        if (P.variant == RAPDB_YX) {
          step = gf + gt;
        } else {
          I.gx[S.gxcur][j] = grad;
          const double gprev = (k == 0) ? grad : I.gx[S.gxcur ^ 1][j];
          step = (1.0 + theta) * grad - theta * gprev;
        }
        const double lo = I.lb[j], hi = I.ub[j];
        if (I.hyp_a) keep_for_projection(xj - tau * step);     // finished in phase HYPX
        else trial_final(fmin(fmax(xj - tau * step, lo), hi), u0);
        if (gap_due && S.gap_evals == 0) I.gpf[j] = hash_unit((uint32_t)j);
        if (fresh) {
          if (P.log_cap > 0 && it >= 1 && it <= P.log_cap && P.x_log)
            P.x_log[(size_t)(it - 1) * n + j] = (float)xj;
          if (P.restart_from_average && k >= 1)
            I.xcum[j] = (k == 1 ? 0.0 : I.xcum[j]) + S.t_last * xj;
        }
      }
    } else if (phase == PH_GAPP) {
      // power iteration on Q(y): consume Q(y)p of the last pass, write the next p
      const float pj = I.gpf[j];
      const double hp = (I.s_off ? q0d * (double)pj : (double)Un[j]) + gc;
      acc[V_AA] = (double)pj * hp;
      acc[V_BB] = (double)pj * (double)pj;
      acc[V_X2] = hp * hp;
      if (gap_iter < gap_P) {
        const float pn = (float)(hp / S.gap_pnorm);
        I.gpf[j] = pn;
        sx[lc] = pn;
        sd[lc] = pn;
      } else {
        // last power step: the accelerated gradient starts at z_0 = w_0 = x^k
        I.gz[j] = xj;
        I.gzf[j] = xj32;
        I.gwf[j] = xj32;
        sx[lc] = xj32;
        sd[lc] = xj32;
      }
    } else if (phase == PH_GAPF || phase == PH_GAPV) {
      // x-subproblem min_{z in X} Phi(z, y) + xi |z - x|^2 (Hessian Q(y) + 2 xi I)
      const float zk32 = I.gzf[j];
      const double cl = c0 + g2;                                       // c(y)_j
      const double hz = (I.s_off ? q0d * (double)zk32 : (double)I.W[j]) + gt;  // (Q(y) z)_j
      acc[2] = (double)zk32 * hz;
      acc[3] = cl * (double)zk32;
      acc[4] = ((double)zk32 - xj) * ((double)zk32 - xj);
      if (phase == PH_GAPF) {
        const float wj = I.gwf[j];
        const double hw = (I.s_off ? q0d * (double)wj : (double)Un[j]) + gc;   // (Q(y) w)_j
        const double grad = hw + 2.0 * P.xi * ((double)wj - xj) + cl;
        const double zu = (double)wj - grad / S.gap_L;
        if (I.hyp_a) keep_for_projection(zu);                         // finished in phase HYPX
        else gapf_final(fmin(fmax(zu, (double)I.lb[j]), (double)I.ub[j]));
      }
    } else if (phase == PH_XY2) {
      // a = sum_i dy_i (u~_i + c_i),  b = Q(y^k) d = w_0 + sum_i y_i w_i
      const double bb = (double)I.W[j] + gt;
      acc[V_AA] = gc * gc;
      acc[V_BB] = bb * bb;
    } else if (phase == PH_INIT || phase == PH_AVG) {
      // the new start point: x^0 itself, or the weighted average of the run
      const double xt = (phase == PH_INIT) ? xj : I.xcum[j] / S.T;
      const float xt32 = (float)xt;
      xt_out[j] = xt;
      xt_out32[j] = xt32;
      xt_outlo[j] = (float)(xt - (double)xt32);
      I.dv[j] = 0.0f;
      sx[lc] = xt32;
      sd[lc] = 0.0f;
      if (I.s_off) {
        const float u0n = (float)(q0d * (double)xt32);
        Un[j] = u0n;
        I.W[j] = 0.0f;
        acc[V_XU0] = (double)xt32 * (double)u0n;
      }
      acc[V_CX0] = c0 * (double)xt32;
    }
  }
  // (with the hyperplane the trial and gradient-step right-hand sides are
  // written in phase HYPX, after the projection)
  if (ST == RAPDB_FP8 && ((phase == PH_TRIAL && (!I.hyp_a || gap_due)) || phase == PH_INIT || phase == PH_AVG ||
                           phase == PH_GAPP || (phase == PH_GAPF && !I.hyp_a) || phase == PH_HYPX)) {
    // pre-scaled right-hand sides s_i .* (first, second right-hand side) of every stored matrix
    __syncthreads();
    if (j < n) {
      float xv = sx[lc], dvv = sd[lc];
      if (phase == PH_TRIAL && gap_due && grp >= 0) {
        // the trial may be replaced by the first power pass: its RHS is p_0
        xv = I.gpf[j];
        dvv = xv;
      }
      for (int s = grp; s < I.M; s += NGRP) {
        const float sc = I.qscale[(size_t)s * ldv + j];
        XS[(size_t)s * ldv + j] = sc * xv;
        VS[(size_t)s * ldv + j] = sc * dvv;
      }
    }
  }
  if (cb == 0 && tid == 0 && fresh && phase == PH_TRIAL && P.log_cap > 0 && it >= 1 && it <= P.log_cap &&
      P.y_log) {
    for (int i = 0; i < m; ++i) P.y_log[(size_t)(it - 1) * m + i] = (float)ys[i];
  }

  // every column's partials are in warp 0 (constraint group 0): a warp sum
  // in a fixed order suffices
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < NVP; ++q) acc[q] = warp_sum(acc[q]);
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < NVP; ++q) I.vpart[(size_t)cb * NVP + q] = acc[q];
    }
  }
  if (!arrive_last(&states[b].arrive_vec, (unsigned)I.ncb)) return;

  // ---- last CTA of this instance: the control step, on a shared-memory copy
  // of the state (its serial scalar updates then cost no global round trips;
  // written back at the end) ----
  __syncthreads();   // (every thread has read its copy of the state above)
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&states[b]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&Sc);
    for (int w = tid; w < (int)(sizeof(State) / 4); w += NT) dst[w] = src[w];
  }
  __syncthreads();
  // (every barrier below is reached by all threads before any of them leaves)
  auto control = [&](State& S) {

    // ---- last CTA of this instance: fixed-order reduction + control ----
    // (one warp per partial slot, lanes striding over the column blocks)
    {
      const int lane = tid & 31, warp = tid >> 5;
      for (int q = warp; q < NVP; q += NWARP) {
        double s = 0.0;
#pragma unroll 4
        for (int bq = lane; bq < I.ncb; bq += 32) s += __ldcg(&I.vpart[(size_t)bq * NVP + q]);
        s = warp_sum(s);
        if (lane == 0) vfin[q] = s;
      }
    }
    __syncthreads();

    const bool hyp_trial_x = phase == PH_HYPX && S.hyp_ret == PH_TRIAL;
    if (phase == PH_INIT || phase == PH_AVG || (phase == PH_TRIAL && !I.hyp_a) || hyp_trial_x) {
      if (tid == 0) {
        S.dd = vfin[V_DD];
        for (int q = 0; q < NDOT; ++q) S.dots0[q] = vfin[V_XU0 + q];
        if (phase == PH_AVG) S.phase = PH_AVGP;   // the pass of this body forms U = Q xbar
      }
    }
    if (hyp_trial_x) {              // the projected trial point is ready for the pass
      if (tid == 0) {
        S.phase = PH_TRIAL;
        S.trial_ready = 1;
      }
      return;
    }
    // shared scratch of the hyperplane routines (red holds NWARP * NVP doubles)
    float2* hsm = reinterpret_cast<float2*>(red);
    double* hsb = red + NWARP + 2;
    if (phase == PH_TRIAL && fresh) {
      double fe[2] = {0.0, 0.0};
      double rs2 = vfin[V_RS];
      if (kkt_due) {
        kkt_feas_terms(I, gk, ys, fe[0], fe[1], red);
        block_allsum<2>(fe, red);
        if (I.hyp_a) {   // dist(0, grad + N_X(x^k)) with the hyperplane's direction
          double t_new;
          rs2 = hyp_cone_rs2(I, I.xf[S.xcur], I.xl[S.xcur], S.hyp_t, &t_new, hsm, hsb);
          if (tid == 0) S.hyp_t = t_new;
        }
      }
      if (tid != 0) return;
      if (kkt_due) {
        double rel, rs, rf;
        kkt_finish(I, rs2, vfin[V_GF], vfin[V_GC], fe[0], fe[1], rel, rs, rf);
        S.rel_kkt = rel;
        S.r_stat = rs;
        S.r_feas = rf;
        if (P.kkt_log && it < P.log_cap) P.kkt_log[it] = rel;
        if (!(rel == rel)) { finish(S, ctrl, RAPDB_ERR_NUMERIC); return; }
        if (can_refine(I, S)) {
          S.rel_q = rel;
          // the check runs at this x^k, after the stored level's residual at
          // the same point (rel_q) has been formed
          if (rel <= P.tol || S.check_due) {
            S.check_due = 0;
            start_check(I, S);
            return;
          }
        } else if (rel <= P.tol) {
          finish(S, ctrl, RAPDB_OK);
          return;
        }
      }
      if (it >= P.max_iter) { finish(S, ctrl, RAPDB_ERR_MAXITER); return; }
      if (S.deadline_ns > 0 && (long long)globaltimer() > S.deadline_ns) {
        finish(S, ctrl, RAPDB_ERR_TIMEOUT);
        return;
      }
      if (S.avg_pending) {          // restart from the average: the trial is discarded
        S.avg_pending = 0;
        S.fresh = 0;
        S.phase = PH_AVG;
        return;
      }
      if (gap_due) {                // smoothed-gap evaluation first: the trial is discarded
        S.fresh = 0;
        S.gap_it_done = it;
        S.gap_iter = 1;             // the pass of this body is power pass #1 (right-hand side p_0)
        S.gap_pnorm = 1.0;
        S.phase = PH_GAPP;
        return;
      }
      S.restarts += S.restart_note;
      S.restart_note = 0;
      S.fresh = 0;
      if (I.hyp_a) {                // the trial point is projected onto X first
        S.hyp_ret = PH_TRIAL;
        S.phase = PH_HYPN;
      } else {
        S.trial_ready = 1;
      }
      return;
    }
    if (phase == PH_TRIAL) {        // a further trial of the same iteration
      if (tid == 0) {
        if (I.hyp_a) {
          S.hyp_ret = PH_TRIAL;
          S.phase = PH_HYPN;
        } else {
          S.trial_ready = 1;
        }
      }
      return;
    }
    if (phase == PH_GAPP) {
      if (gap_iter == 1) {
        // y-part of G_xi in closed form, y' = proj_Y(y + g(x)/(2 xi)) (max(0, .), or
        // the simplex projection): fixed during the evaluation
        for (int i = tid; i < m; i += NT) {
          const double v = ys[i] + gk[i] / (2.0 * P.xi);
          yts[i] = (P.dual_simplex || i >= I.m_ineq) ? v : fmax(0.0, v);
        }
        __syncthreads();
        if (P.dual_simplex) proj_simplex_block(yts, I.m_ineq, P.dual_r, red);
        double yp[2] = {0.0, 0.0};
        for (int i = tid; i < m; i += NT) {
          const double lp = yts[i];
          yp[0] += lp * gk[i];
          yp[1] += (lp - ys[i]) * (lp - ys[i]);
        }
        block_allsum<2>(yp, red);
        if (tid == 0) S.gap_ypart = S.obj + yp[0] - P.xi * yp[1];
      }
      if (tid != 0) return;
      const double mu = vfin[V_AA] / vfin[V_BB];
      S.gap_pnorm = sqrt(vfin[V_X2]);
      if (!(S.gap_pnorm > 0.0) || !(mu == mu)) S.gap_pnorm = 1.0;
      if (gap_iter < gap_P) {
        S.gap_iter = gap_iter + 1;
        return;
      }
      // step constant of the accelerated gradient: L = 2 mu + 2 xi (the
      // Rayleigh quotient mu bounds lambda_max(Q(y)) from below), constant
      // momentum (sqrt(L) - sqrt(2 xi)) / (sqrt(L) + sqrt(2 xi)) for the
      // 2 xi-strongly convex subproblem
      const double lq = fmax(mu, 0.0);
      S.gap_L = 2.0 * lq + 2.0 * P.xi;
      const double sl = sqrt(S.gap_L), sm = sqrt(2.0 * P.xi);
      S.gap_mu = (sl - sm) / (sl + sm);
      S.gap_beta = S.gap_mu;
      S.gap_prev = INFINITY;
      S.gap_iter = 0;
      S.phase = PH_GAPF;
      return;
    }
    if (phase == PH_GAPF || phase == PH_GAPV || phase == PH_HYPX) {
      // x-subproblem objective at z_k: 0.5 z'Q(y)z + c(y)'z + y'd + xi |z - x|^2
      double xval;
      if (phase == PH_HYPX) {
        xval = S.gap_xval;          // formed before the projection of the step
      } else {
        double yd[1] = {0.0};
        for (int i = tid; i < m; i += NT) yd[0] += ys[i] * I.dcon[i];
        block_allsum<1>(yd, red);
        xval = 0.5 * vfin[2] + vfin[3] + yd[0] + P.xi * vfin[4];
      }
      if (phase == PH_GAPF && I.hyp_a) {   // the step is projected onto X first
        if (tid == 0) {
          S.gap_xval = xval;
          S.hyp_ret = PH_GAPF;
          S.phase = PH_HYPN;
        }
        return;
      }
      if (phase == PH_GAPF || phase == PH_HYPX) {
        if (tid != 0) return;
        if (phase == PH_HYPX) S.phase = PH_GAPF;
        // function-value restart of the momentum: after an increase of the
        // subproblem objective the next step is a plain projected gradient step
        S.gap_beta = (gap_iter > 0 && xval > S.gap_prev) ? 0.0 : S.gap_mu;
        S.gap_prev = xval;
        const int k1 = gap_iter + 1;
        const bool small = vfin[0] <= 1e-20 * (1.0 + vfin[1]);
        // objective error bound of the strongly convex subproblem from the
        // gradient mapping L (w - z+): <= L^2 |z+ - w|^2 / (2 * 2 xi); the
        // restart rule compares G with q G_ref, so 1e-3 of the current gap
        // estimate suffices
        const double err = S.gap_L * S.gap_L * vfin[5] / (4.0 * P.xi);
        const double gest = S.gap_ypart - xval;
        const bool accurate = gap_iter >= 3 && gest > 0.0 && err <= 1e-3 * gest + 1e-13 * (1.0 + fabs(xval));
        if (k1 >= P.gap_inner_max || small || accurate) {
          S.phase = PH_GAPV;       // the pass of this body forms Q z_K
        } else {
          S.gap_iter = k1;
        }
        return;
      }
      // PH_GAPV: G = y-part (closed form, computed at the first power step) - x-part
      if (tid != 0) return;
      const double G = S.gap_ypart - xval;
      S.gap_val = G;
      if (P.gap_log && S.gap_evals < P.log_cap) P.gap_log[S.gap_evals] = G;
      S.gap_evals += 1;
      bool fire = false;
      if (!S.gap_has_ref) {
        S.gap_ref = G;
        S.gap_has_ref = 1;
      } else if (G <= P.q * S.gap_ref) {
        fire = true;
        S.gap_ref = G;
      }
      S.gap_iter = 0;
      S.phase = PH_TRIAL;          // the next body's vector kernel prepares the trial
      if (fire) {
        restart_scalars(P, S);
        S.restarts += 1;
        if (can_refine(I, S) && S.precision < 2) {
          S.fresh = 1;
          S.check_due = 1;
        }
      }
      return;
    }
    if (phase == PH_XY2) {
      double dy2[1] = {0.0};
      for (int i = tid; i < m; i += NT) { const double t = yts[i] - ys[i]; dy2[0] += t * t; }
      block_allsum<1>(dy2, red);
      const double sig = sigma, an = P.c_alpha / tau, bn = P.gamma0 * P.c_beta / sig;
      const int k0 = S.k;
      const double t_acc = sig / (k0 == 0 ? sig : S.sigma0);
      if (tid == 0) {
        const double ddy = 0.5 * dy2[0];
        const double dp = 0.5 * S.dd;
        const double bterm = (bn > 0.0) ? vfin[V_BB] / (2.0 * bn) : (vfin[V_BB] == 0.0 ? 0.0 : INFINITY);
        const double E = vfin[V_AA] / (2.0 * an) - ddy / sig + bterm - (1.0 / tau - theta * (S.alpha_k + S.beta_k)) * dp;
        const bool ok = E <= -P.delta / tau * dp - P.delta / sig * ddy;
        S.trials_total += 1;
        s_dec = !(E == E) ? 2 : ((ok || !P.backtracking) ? 1 : 0);
      }
      __syncthreads();
      const int dec = s_dec;
      if (dec == 1) {
        accept_vectors(I, k0, gcur0, ycur0, t_acc);
        __syncthreads();
        if (tid == 0) accept_scalars(I, S, sig, an, bn);
      } else if (tid == 0) {
        if (dec == 2) finish(S, ctrl, RAPDB_ERR_NUMERIC);
        else reject_trial(I, S, ctrl);
      }
      return;
    }
    if (phase == PH_KKT32B) {
      // the residual one precision level up (check_level) at x^k
      double fe[2] = {0.0, 0.0};
      kkt_feas_terms(I, I.gnew, ys, fe[0], fe[1], red);
      block_allsum<2>(fe, red);
      double rs2 = vfin[V_RS];
      if (I.hyp_a) {
        double t_new;
        rs2 = hyp_cone_rs2(I, I.xf[S.xcur], I.xl[S.xcur], S.hyp_t, &t_new, hsm, hsb);
        if (tid == 0) S.hyp_t = t_new;
      }
      if (tid == 0) {
        double rel, rs, rf;
        kkt_finish(I, rs2, vfin[V_GF], vfin[V_GC], fe[0], fe[1], rel, rs, rf);
        S.rel_kkt = rel;
        S.r_stat = rs;
        S.r_feas = rf;
        int dec = 0;
        if (rel <= P.tol) {
          dec = 2;
        } else {
          if (S.precision == 3) {
            // the quantised-increment level: every check re-anchors U, so the
            // storage error cannot build up beyond ANCHOR_EVERY iterations and
            // shrinks with the steps.  Checks come every ANCHOR_EVERY
            // iterations, too often for the halving test (the residual of the
            // method is not monotone, and it can sit on a plateau for
            // thousands of iterations at float32 as well): kkt_ref is the
            // lowest true residual so far, and the level switches when four
            // checks in a row find none lower while the level's own residual
            // at the same point (rel_q) misses the true one by more than half
            // of it, i.e. when the stall is the storage's and not the
            // method's.  A check that the drifted products' residual triggered
            // (rel_q <= tol) and that finds the true one above tol re-anchors
            // and the level carries on
            if (S.kkt_ref > 0.0 && rel >= S.kkt_ref) {
              S.stall_count += 1;
            } else {
              S.stall_count = 0;
              S.kkt_ref = rel;
            }
            if (S.stall_count >= 4 && fabs(S.rel_q - rel) > 0.5 * rel) dec = 1;
          } else {
            const bool stalled = (S.kkt_ref > 0.0 && rel > P.stall_ratio * S.kkt_ref);
            S.kkt_ref = rel;
            // switch when the true residual stalls, when the stored matrices'
            // problem is solved, or when the storage error already dominates
            // (the true residual is more than twice the stored level's)
            if (stalled || S.rel_q <= P.tol || rel > 2.0 * S.rel_q) dec = 1;
          }
        }
        s_dec = dec;
      }
      __syncthreads();
      const int dec = s_dec;
      // the check pass output becomes the current U on a switch, and at level 3
      // always (the check is its anchor)
      const bool adopt = dec == 1 || (dec == 0 && S.precision == 3);
      if (adopt) {   // (row 0 of a Q_0 that is not stored was formed above, at x^k)
        double* gd = I.gb[gcur0];
        for (int i = tid; i < m; i += NT) gd[i] = I.gnew[i];
        __syncthreads();
      }
      if (tid == 0) {
        if (dec == 2) {
          finish(S, ctrl, RAPDB_OK);
        } else {
          if (dec == 1) {
            // the products' precision changes, the iteration's state does not:
            // step sizes, momentum and the counter carry on from x^k (a check
            // at a restart boundary follows the restart that happened there)
            S.precision = S.check_level;
            S.switches += 1;
            if (S.switch_it < 0) S.switch_it = S.it;
          }
          if (adopt) {
            S.ucur ^= 1;
            S.anchor_age = 0;       // the check pass formed U directly
          }
          S.fresh = 1;
          S.phase = PH_TRIAL;
        }
      }
      return;
    }
  };
  control(Sc);
  __syncthreads();
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&Sc);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&states[b]);
    for (int w = tid; w < (int)(sizeof(State) / 4); w += NT) dst[w] = src[w];
  }
}

// ---------------------------------------------------------------------------
// Projection onto X with the hyperplane (phase HYPN): the scalar nu of
// x = clamp(v - nu a) with a'x = beta, on one CTA of NTH threads; the vector
// kernel of phase HYPX then forms x column by column.
// ---------------------------------------------------------------------------
constexpr int NTH = 1024;
template <int DUMMY>
__global__ void __launch_bounds__(NTH) k_hyp(const Inst* __restrict__ insts, State* __restrict__ states) {
  __shared__ float2 sm[NTH / 32 + 2];
  __shared__ double sb[2];
  const Inst& I = insts[0];
  State& S = states[0];
  if (S.phase != PH_HYPN) return;
  const double nu = hyp_proj_nu(I, S.hyp_nu, sm, sb);
  if (threadIdx.x == 0) {
    S.hyp_nu = nu;
    S.phase = PH_HYPX;
  }
}

// ---------------------------------------------------------------------------
// Tile variant of the coupling pass: NST == 0 streams Q through registers
// (RPW rows x UNR 16-byte chunks in flight per lane); NST > 0 stages Q through
// shared memory with bulk copies: per warp (NST slots of CWB bytes per row,
// RPW > 0), or per CTA in whole-row stages of CWB bytes (RPW == 0).
// ---------------------------------------------------------------------------
// dynamic shared memory of a bulk-copy variant: the warps' mbarriers (8 bytes
// each, area rounded up to 128 bytes) followed by the slot buffers
template <int NST>
__host__ __device__ constexpr size_t tma_bar_bytes() {
  return NST <= 0 ? 0 : ((size_t)NWARP * (size_t)(NST > 0 ? NST : 0) * 8 + 127) / 128 * 128;
}
template <int NST, int RPW, int CWB>
__host__ __device__ constexpr size_t tma_smem_bytes() {
  return NST <= 0 ? 0 : (RPW == 0 ? rows_smem_bytes<CWB, NST>() : tma_bar_bytes<NST>() + (size_t)NWARP * NST * RPW * CWB);
}

// Rows per warp of the float32 products inside a kernel of storage ST: the
// float32 refinement copy of a quantised matrix keeps four rows per warp.
template <int ST, int RPW>
constexpr int F32_RPW = (ST == RAPDB_F32 || RPW <= 4) ? RPW : 4;
// Rows per warp and chunks in flight of the incremental compensated pass
// (register streaming): the tile's own where it streams through registers.
template <int ST, int RPW>
constexpr int INC_RPW = (RPW == 0) ? 4 : F32_RPW<ST, RPW>;
template <int UNR>
constexpr int INC_UNR = (UNR == 0) ? 2 : UNR;

template <int ST, int RPW, int UNR, int NST, int CWB>
__device__ __forceinline__ void pass_tile(const uint8_t* Qm, int ld, int row0, int rows, const float* x,
                                          const float* v, const float* xs, const float* vs, const float* scale,
                                          const float* uold, const float* crow, float* Uo, float* Wo, double* out,
                                          int ostride, double* red, uint8_t* dsm, int* err) {
  if constexpr (NST == 0) {
    pass_block<ST, RPW, UNR>(Qm, ld, row0, rows, x, v, xs, vs, scale, uold, crow, Uo, Wo, out, ostride, red);
  } else if constexpr (NST < 0) {
    pass_block_pipe<ST, RPW, UNR>(Qm, ld, row0, rows, x, v, xs, vs, scale, uold, crow, Uo, Wo, out, ostride, red);
  } else if constexpr (RPW == 0) {
    // whole-row stages of CWB bytes; rows longer than a stage stream through registers
    if ((size_t)ld * Elt<ST>::B <= (size_t)CWB)
      pass_block_rows<ST, CWB, NST>(Qm, ld, row0, rows, x, v, xs, vs, scale, uold, crow, Uo, Wo, out, ostride, red,
                                    dsm, err);
    else
      pass_block<ST, 4, 4>(Qm, ld, row0, rows, x, v, xs, vs, scale, uold, crow, Uo, Wo, out, ostride, red);
  } else {
    uint64_t* bars = reinterpret_cast<uint64_t*>(dsm);
    uint8_t* sbuf = dsm + tma_bar_bytes<NST>();
    pass_block_tma<ST, RPW, NST, CWB>(Qm, ld, row0, rows, x, v, xs, vs, scale, uold, crow, Uo, Wo, out, ostride,
                                      red, sbuf, bars, err);
  }
}

// ---------------------------------------------------------------------------
// k_pass: the fused coupling pass + post-control
// ---------------------------------------------------------------------------
static __device__ void pass_finish(const Inst& I, State& S, Ctrl* ctrl, int s, int i, const double* part, int nb,
                                   int phase, bool comp, const float* x, const float* v, double* red, int& s_dec);
static __device__ void pass_control(const Inst& I, State& S, Ctrl* ctrl, int phase, bool comp, const float* x,
                                    const float* v, double* red, int& s_dec, double* Dsh = nullptr);

template <int ST, int RPW, int UNR, int NST, int CWB>
__device__ __forceinline__ void pass_body(const Inst* __restrict__ insts, State* __restrict__ states,
                                          Ctrl* __restrict__ ctrl, const int* __restrict__ pmap,
                                          const float* __restrict__ XS, const float* __restrict__ VS, uint8_t* dsm,
                                          double* red, int& s_dec, int bid) {
  const int b = pmap[bid];
  const Inst& I = insts[b];
  State& S = states[b];
  const int phase = S.phase;
  if (!pass_phase(phase)) return;
  if (phase == PH_TRIAL && !S.trial_ready) return;   // no trial prepared in this body
  const int item = bid - I.pblk0;
  const int s = item / I.nrb;
  const int r = item - s * I.nrb;
  const int i = s + I.s_off;
  const int row0 = r * I.rb;
  const int rows = min(I.rb, I.n - row0);
  const int ldv = I.ldv;
#ifdef RAPDB_CHECKED
  {
    const bool in_range = item >= 0 && item < I.M * I.nrb && rows >= 1 && rows <= I.rb && i <= I.m_ineq;
    const int code = !in_range ? CHK_PASS_RANGE
                     : (NST > 0 && dyn_smem_bytes() < (unsigned)tma_smem_bytes<NST, RPW, CWB>() ? CHK_PASS_SMEM : 0);
    if (code) {
      if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, code);
      return;
    }
  }
#endif
  const int level = (phase == PH_KKT32) ? S.check_level : S.precision;
  const bool comp = (level >= 2) && !gap_phase(phase);               // compensated products
  const bool use32 = (ST != RAPDB_F32) && (level >= 1);
  const bool at_xk = phase == PH_KKT32 || phase == PH_ANCHOR;       // products at the accepted iterate
  const float* x;
  const float* v;
  if (at_xk) {
    x = I.xf[S.xcur];
    v = x;
  } else if (phase == PH_GAPP) {
    x = I.gpf;
    v = x;
  } else if (phase == PH_GAPF || phase == PH_GAPV) {
    x = I.gwf;
    v = I.gzf;
  } else {
    x = I.xf[S.xcur ^ 1];
    v = I.dv;
  }
  const float* uold = (at_xk || gap_phase(phase)) ? nullptr : I.U[S.ucur] + (size_t)i * ldv;
  float* Uo = I.U[S.ucur ^ 1] + (size_t)i * ldv;
  float* Wo = I.W + (size_t)i * ldv;
  double* out = I.part + (size_t)s * NDOT * I.nrb + r;
  const float* crow = I.c + (size_t)i * ldv;
  if (comp) {
    const float* Qb = (ST == RAPDB_F32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32) ? I.ld : I.ld32;
    const float* xlo = at_xk ? I.xl[S.xcur] : I.xl[S.xcur ^ 1];
    if (phase == PH_TRIAL)   // U' = U^k + Q d
      pass_block_incr<INC_RPW<ST, RPW>, INC_UNR<UNR>>(Qb + (size_t)s * I.n * ldq, ldq, row0, rows, x, xlo, v, uold,
                                                     I.Ulo[S.ucur] + (size_t)i * ldv, crow, Uo,
                                                     I.Ulo[S.ucur ^ 1] + (size_t)i * ldv, Wo, out, I.nrb, red);
    else
      pass_block_prec2<4, 2>(Qb + (size_t)s * I.n * ldq, ldq, row0, rows, x, xlo, v, uold,
                             uold ? I.Ulo[S.ucur] + (size_t)i * ldv : nullptr, crow, Uo,
                             I.Ulo[S.ucur ^ 1] + (size_t)i * ldv, Wo, out, I.nrb, red);
  } else if (use32 || ST == RAPDB_F32) {
    const float* Qb = (ST == RAPDB_F32 && !use32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32 && !use32) ? I.ld : I.ld32;
    pass_tile<RAPDB_F32, F32_RPW<ST, RPW>, UNR, NST, CWB>((const uint8_t*)(Qb + (size_t)s * I.n * ldq), ldq, row0,
                                                         rows, x, v, nullptr, nullptr, nullptr, uold, crow, Uo, Wo,
                                                         out, I.nrb, red, dsm, &ctrl->err);
  } else {
    constexpr int EB = Elt<ST>::B;
    const uint8_t* Qb = (const uint8_t*)I.Q + (size_t)s * I.n * I.ld * EB;
    pass_tile<ST, RPW, UNR, NST, CWB>(Qb, I.ld, row0, rows, x, v, XS ? XS + (size_t)s * ldv : nullptr,
                                      VS ? VS + (size_t)s * ldv : nullptr,
                                      I.qscale ? I.qscale + (size_t)s * ldv : nullptr, uold, crow, Uo, Wo, out,
                                      I.nrb, red, dsm, &ctrl->err);
  }
  pass_finish(I, S, ctrl, s, i, I.part, I.nrb, phase, comp, x, v, red, s_dec);
}

template <int ST, int RPW, int UNR, int NST, int CWB>
__global__ void __launch_bounds__(NT, (NST <= 0 ? 2 : 1)) k_pass(const Inst* __restrict__ insts,
                                                                State* __restrict__ states,
                                                                Ctrl* __restrict__ ctrl, const int* __restrict__ pmap,
                                                                const float* __restrict__ XS,
                                                                const float* __restrict__ VS) {
  extern __shared__ __align__(128) uint8_t dsm[];
  __shared__ double red[NWARP * NDOT];
  __shared__ int s_dec;
  pass_body<ST, RPW, UNR, NST, CWB>(insts, states, ctrl, pmap, XS, VS, dsm, red, s_dec, blockIdx.x);
}

// After a CTA's share of a pass: the last arrival of matrix s reduces the
// matrix's nb row-block dot partials (part, (M, NDOT, nb)) in a fixed order;
// the last matrix of the instance runs the control step of the phase.
static __device__ void pass_finish(const Inst& I, State& S, Ctrl* ctrl, int s, int i, const double* part, int nb,
                                   int phase, bool comp, const float* x, const float* v, double* red, int& s_dec) {
  if (!arrive_last(&I.mcount[s], (unsigned)nb)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < NDOT) {
    const double* src = part + ((size_t)s * NDOT + warp) * nb;
    double t = 0.0;
#pragma unroll 4
    for (int rr = lane; rr < nb; rr += 32) t += __ldcg(src + rr);
    t = warp_sum(t);
    if (lane == 0) I.dots[(size_t)i * NDOT + warp] = t;
  }
  // ---- last matrix of the instance: control ----
  if (!arrive_last(&S.arrive_pass, (unsigned)I.M)) return;
  pass_control(I, S, ctrl, phase, comp, x, v, red, s_dec);
}

// The control step after a pass, on one CTA, once every matrix's dots are in
// I.dots: the equality dots, g at the pass point, and the phase's decision
// (the yx backtracking test and step rule, the xy dual step, or the set-up,
// restart, check and anchor bookkeeping).
// Dsh: the reduced dots in shared memory (the packed pass's control kernel
// formed them there), else they are read from I.dots, bypassing L1.
static __device__ void pass_control(const Inst& I, State& S, Ctrl* ctrl, int phase, bool comp, const float* x,
                                    const float* v, double* red, int& s_dec, double* Dsh) {
  const int tid = threadIdx.x;
  auto dl = [Dsh](const double* p) { return Dsh ? *p : __ldcg(p); };
  const int ldv = I.ldv;
  if (I.s_off && tid < NDOT) {
    I.dots[tid] = S.dots0[tid];
    if (Dsh) Dsh[tid] = S.dots0[tid];
  }
  if (I.m > I.m_ineq && !gap_phase(phase)) {
    // linear equalities (no stored matrix): u = w = 0, c'x and c'v here
    const float* xlo_e =
        comp ? ((phase == PH_KKT32 || phase == PH_ANCHOR) ? I.xl[S.xcur] : I.xl[S.xcur ^ 1]) : nullptr;
    for (int ie = I.m_ineq + 1; ie <= I.m; ++ie) {
      const float* ci = I.c + (size_t)ie * ldv;
      double sv[2] = {0.0, 0.0};
      for (int jj = tid; jj < I.n; jj += NT) {
        const double xj = (double)x[jj] + (xlo_e ? (double)xlo_e[jj] : 0.0);
        sv[0] += (double)ci[jj] * xj;
        sv[1] += (double)ci[jj] * (double)v[jj];
      }
      block_allsum<2>(sv, red);
      if (tid == 0) {
        for (int c2 = 0; c2 < (Dsh ? 2 : 1); ++c2) {
          double* Di = (c2 ? Dsh : I.dots) + (size_t)ie * NDOT;
          Di[D_XU] = 0.0;
          Di[D_VW] = 0.0;
          Di[D_VUO] = 0.0;
          Di[D_CX] = sv[0];
          Di[D_CV] = sv[1];
        }
      }
    }
  }
  __syncthreads();

  const DevParams& P = I.P;
  const int m = I.m;
  const double* D = Dsh ? Dsh : I.dots;
  const int k0 = S.k, gcur0 = S.gcur, ycur0 = S.ycur;
  if (gap_phase(phase)) {          // smoothed-gap passes: the vector kernel consumes the products
    if (tid == 0) S.passes += 1;
    return;
  }
  if (phase == PH_TRIAL && tid == 0) S.trial_ready = 0;
  // g at the pass point: g_i = 0.5 x'Q_i x + c_i'x + d_i, with the per-phase
  // per-constraint work fused into the same loop
  if (phase == PH_TRIAL && P.variant == RAPDB_YX) {
    const double tau = S.tau;
    const double sig = S.gamma * tau;
    const double th = S.sigma_prev / sig;
    const double* yt = I.yb[ycur0 ^ 1];
    const double* y = I.yb[ycur0];
    double acc[3] = {0.0, 0.0, 0.0};   // sum y~_i d'Q_i d, |dg|^2, |dy|^2
    for (int ii = tid; ii < m; ii += NT) {
      const double* Di = D + (size_t)(ii + 1) * NDOT;
      const double vw = dl(&Di[D_VW]);
      I.gnew[ii] = 0.5 * dl(&Di[D_XU]) + dl(&Di[D_CX]) + I.dcon[ii];
      acc[0] += yt[ii] * vw;
      const double dgi = dl(&Di[D_VUO]) + dl(&Di[D_CV]) + 0.5 * vw;
      acc[1] += dgi * dgi;
      const double t = yt[ii] - y[ii];
      acc[2] += t * t;
    }
    block_allsum<3>(acc, red);
    const double an = P.c_alpha / sig;
    const double t_acc = sig / (k0 == 0 ? sig : S.sigma0);
    if (tid == 0) {
      const double dQd = dl(&D[D_VW]) + acc[0];
      const double E = 0.5 * dQd - S.dd / (2.0 * tau) + acc[1] / (2.0 * an) - (1.0 / sig - th * S.alpha_k) * 0.5 * acc[2];
      const bool ok = E <= -P.delta * S.dd / (2.0 * tau) - P.delta * acc[2] / (2.0 * sig);
      S.trials_total += 1;
      S.passes += 1;
      s_dec = !(E == E) ? 2 : ((ok || !P.backtracking) ? 1 : 0);
    }
    __syncthreads();
    const int dec = s_dec;
    if (dec == 1) {
      accept_vectors(I, k0, gcur0, ycur0, t_acc);
      __syncthreads();
      if (tid == 0) accept_scalars(I, S, sig, an, 0.0);
    } else if (tid == 0) {
      if (dec == 2) finish(S, ctrl, RAPDB_ERR_NUMERIC);
      else reject_trial(I, S, ctrl);
    }
    return;
  }
  if (phase == PH_TRIAL) {
    // xy: dual ascent at the new primal point, then the a/b sweep
    const double sig = S.gamma * S.tau;
    const double* y = I.yb[ycur0];
    double* yt = I.yb[ycur0 ^ 1];
    for (int ii = tid; ii < m; ii += NT) {
      const double* Di = D + (size_t)(ii + 1) * NDOT;
      const double g = 0.5 * dl(&Di[D_XU]) + dl(&Di[D_CX]) + I.dcon[ii];
      I.gnew[ii] = g;
      yt[ii] = (P.dual_simplex || ii >= I.m_ineq) ? y[ii] + sig * g : fmax(0.0, y[ii] + sig * g);
    }
    __syncthreads();
    if (P.dual_simplex) proj_simplex_block(yt, I.m_ineq, P.dual_r, red);
    if (tid == 0) {
      S.passes += 1;
      S.phase = PH_XY2;
    }
    return;
  }
  // INIT / AVGP / KKT32 / ANCHOR: g at the pass point
  double* gd = I.gb[gcur0];
  const double T0 = S.T;
  for (int ii = tid; ii < m; ii += NT) {
    const double* Di = D + (size_t)(ii + 1) * NDOT;
    const double g = 0.5 * dl(&Di[D_XU]) + dl(&Di[D_CX]) + I.dcon[ii];
    I.gnew[ii] = g;
    if (phase != PH_KKT32) gd[ii] = g;
    if (phase == PH_AVGP) I.yb[ycur0][ii] = I.ycum[ii] / T0;
  }
  if (phase == PH_ANCHOR && I.s_off) {
    // Q_0 is not stored: its row of U (q0 .* x^k with the low part the
    // vector kernel formed) carries over to the anchored buffer
    const int uc = S.ucur;
    for (int jj = tid; jj < I.n; jj += NT) {
      I.U[uc ^ 1][jj] = I.U[uc][jj];
      if (I.Ulo[0]) I.Ulo[uc ^ 1][jj] = I.Ulo[uc][jj];
    }
  }
  __syncthreads();
  if (tid != 0) return;
  S.passes += 1;
  if (phase == PH_KKT32) {
    S.phase = PH_KKT32B;
    return;
  }
  if (phase == PH_ANCHOR) {
    // the anchored products replace the incremental ones at the same iterate;
    // the iteration's KKT test and restart checks follow (fresh is kept)
    S.ucur ^= 1;
    S.anchor_age = 0;
    S.phase = PH_TRIAL;
    return;
  }
  S.xcur ^= 1;
  S.ucur ^= 1;
  S.anchor_age = 0;         // INIT / AVGP form U directly
  S.obj = 0.5 * dl(&D[D_XU]) + dl(&D[D_CX]);
  if (phase == PH_INIT) {
    S.fresh = 1;
    S.phase = PH_TRIAL;
  } else {
    restart_scalars(P, S);
    S.restarts += 1;
    S.fresh = 0;       // the KKT test of this iteration ran at the last iterate
    S.phase = PH_TRIAL;
  }
}

// ---- stand-alone coupling pass (no control) ------------------------------
// level 0: the stored Q; 1: the float32 Q of a quantised context; 2: float32
// Q with compensated products of x + xlo (low parts of U written to Ulo, the
// uold dot not formed).
template <int ST, int RPW, int UNR, int NST, int CWB>
__global__ void __launch_bounds__(NT, (NST <= 0 ? 2 : 1)) k_pass_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                   const float* __restrict__ v, const float* __restrict__ XS,
                                                   const float* __restrict__ VS, const float* __restrict__ uold,
                                                   float* __restrict__ U, float* __restrict__ W,
                                                   double* __restrict__ part, int level, const float* __restrict__ xlo,
                                                   float* __restrict__ Ulo, int* __restrict__ err) {
  extern __shared__ __align__(128) uint8_t dsm[];
  __shared__ double red[NWARP * NDOT];
  const Inst& I = insts[0];
  const int s = blockIdx.x / I.nrb;
  const int r = blockIdx.x - s * I.nrb;
  const int i = s + I.s_off;
  const int row0 = r * I.rb;
  const int rows = min(I.rb, I.n - row0);
  const int ldv = I.ldv;
#ifdef RAPDB_CHECKED
  if (!(s < I.M && rows >= 1 && rows <= I.rb) ||
      (NST > 0 && dyn_smem_bytes() < (unsigned)tma_smem_bytes<NST, RPW, CWB>())) {
    if (threadIdx.x == 0 && err) atomicCAS(err, 0, CHK_PLAIN_RANGE);
    return;
  }
#endif
  double* out = part + (size_t)s * NDOT * I.nrb + r;
  const float* uo = uold ? uold + (size_t)i * ldv : nullptr;
  const float* crow = I.c + (size_t)i * ldv;
  const int use32 = (ST != RAPDB_F32 && level >= 1) ? 1 : 0;
  if (level == 3) {
    // the incremental form of level 2: U = uold + Q v with uold + Ulo_cur the
    // double-float products at the current iterate
    const float* Qb = (ST == RAPDB_F32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32) ? I.ld : I.ld32;
    pass_block_incr<INC_RPW<ST, RPW>, INC_UNR<UNR>>(Qb + (size_t)s * I.n * ldq, ldq, row0, rows, x, xlo, v, uo,
                                                   I.Ulo[0] + (size_t)i * ldv, crow, U + (size_t)i * ldv,
                                                   Ulo + (size_t)i * ldv, W + (size_t)i * ldv, out, I.nrb, red);
  } else if (level == 2) {
    const float* Qb = (ST == RAPDB_F32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32) ? I.ld : I.ld32;
    // compensated products of x = x + xlo; the low parts of U go to Ulo
    pass_block_prec2<4, 2>(Qb + (size_t)s * I.n * ldq, ldq, row0, rows, x, xlo, v, nullptr, nullptr, crow,
                           U + (size_t)i * ldv, Ulo + (size_t)i * ldv, W + (size_t)i * ldv, out, I.nrb, red);
  } else if (use32 || ST == RAPDB_F32) {
    const float* Qb = (ST == RAPDB_F32 && !use32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32 && !use32) ? I.ld : I.ld32;
    pass_tile<RAPDB_F32, F32_RPW<ST, RPW>, UNR, NST, CWB>((const uint8_t*)(Qb + (size_t)s * I.n * ldq), ldq, row0,
                                                         rows, x, v, nullptr, nullptr, nullptr, uo, crow,
                                                         U + (size_t)i * ldv, W + (size_t)i * ldv, out, I.nrb, red,
                                                         dsm, err);
  } else {
    constexpr int EB = Elt<ST>::B;
    const uint8_t* Qb = (const uint8_t*)I.Q + (size_t)s * I.n * I.ld * EB;
    pass_tile<ST, RPW, UNR, NST, CWB>(Qb, I.ld, row0, rows, x, v, XS ? XS + (size_t)s * ldv : nullptr,
                                      VS ? VS + (size_t)s * ldv : nullptr,
                                      I.qscale ? I.qscale + (size_t)s * ldv : nullptr, uo, crow, U + (size_t)i * ldv,
                                      W + (size_t)i * ldv, out, I.nrb, red, dsm, err);
  }
}

}  // namespace rapdb_dev

#include "rapdb_sym.cuh"
