// Solver kernels of the device-resident rAPDB loop (see rapdb_device.cuh for
// the body structure).  All control decisions are taken on the device by one
// thread of the last-arriving CTA of an instance, in FP64, from partial sums
// reduced in a fixed order (bit-for-bit reproducible runs).
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
  return ph == PH_INIT || ph == PH_TRIAL || ph == PH_XY2 || ph == PH_AVG || ph == PH_KKT32B ||
         ph == PH_GAPY || ph == PH_GAPF;
}
__device__ __forceinline__ bool pass_phase(int ph) {
  return ph == PH_INIT || ph == PH_TRIAL || ph == PH_AVG || ph == PH_KKT32 || ph == PH_GAPY;
}

__device__ __forceinline__ void finish(State& S, Ctrl* ctrl, int status) {
  S.phase = PH_DONE;
  S.status = status;
  atomicSub(&ctrl->active, 1);
}

// Reset of Algorithm 1's initialisation line at a (re)start:
// tau_{-1} = tau_0 = tau_bar, sigma_{-1} = gamma_0 tau_bar, gamma = gamma_0,
// alpha_0 / beta_0 from the parameter recurrences at k = -1.
__device__ void restart_scalars(const DevParams& P, State& S) {
  S.tau_prev = P.tau_bar;
  S.sigma_prev = P.gamma0 * P.tau_bar;
  S.gamma = P.gamma0;
  S.tau = P.tau_bar;
  if (P.variant == RAPDB_YX) {
    S.alpha_k = P.c_alpha / S.sigma_prev;
    S.beta_k = 0.0;
  } else {
    S.alpha_k = P.c_alpha / P.tau_bar;
    S.beta_k = P.gamma0 * P.c_beta / S.sigma_prev;
  }
  S.k = 0;
  S.T = 0.0;
  S.trial = 0;
}

__device__ __forceinline__ bool quantised_refining(const Inst& I, const State& S) {
  return I.storage != RAPDB_F32 && I.P.refine && I.Q32 != nullptr && S.precision == 0;
}

// Relative KKT residual from the reduced partials (thread 0).
__device__ void kkt_from_partials(const Inst& I, const double* g, const double* y, double rs2, double gf2,
                                  double gc2, double& rel, double& r_stat, double& r_feas) {
  double rf2 = 0.0, gd2 = 0.0;
  for (int i = 0; i < I.m; ++i) {
    const double gi = g[i];
    const double ri = (y[i] > 0.0) ? fabs(gi) : fmax(gi, 0.0);
    rf2 += ri * ri;
    const double t = gi - I.dcon[i];
    gd2 += t * t;
  }
  r_stat = sqrt(rs2);
  r_feas = sqrt(rf2);
  const double den_s = 1.0 + fmax(sqrt(gf2), sqrt(gc2));
  const double den_f = 1.0 + fmax(I.dnorm, sqrt(gd2));
  rel = fmax(r_stat / den_s, r_feas / den_f);
}

// Acceptance of the current trial (thread 0): averaging weights, step rule,
// buffer swaps, logging and the fixed-frequency restart rule.
__device__ void accept_trial(const Inst& I, State& S, double sigma, double alpha_next, double beta_next) {
  const DevParams& P = I.P;
  const int nx = S.ycur ^ 1;
  const double tau = S.tau;
  const int trials_this = S.trial + 1;
  if (S.k == 0) S.sigma0 = sigma;
  const double t = sigma / S.sigma0;
  if (P.restart_from_average) {
    const double* yn = I.yb[nx];
    for (int i = 0; i < I.m; ++i) I.ycum[i] = (S.k == 0 ? 0.0 : I.ycum[i]) + t * yn[i];
  }
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
  S.tau_prev = tau;
  S.sigma_prev = sigma;
  S.alpha_k = alpha_next;
  S.beta_k = beta_next;
  S.gamma = gnext;
  S.tau = tnext;
  S.xcur ^= 1;
  S.ycur ^= 1;
  S.ucur ^= 1;
  double* gdst = I.gb[S.gcur ^ 1];
  for (int i = 0; i < I.m; ++i) gdst[i] = I.gnew[i];
  S.gcur ^= 1;
  S.gxcur ^= 1;
  S.k += 1;
  S.it += 1;
  S.trial = 0;
  S.fresh = 1;
  S.obj = 0.5 * I.dots[D_XU] + I.dots[D_CX];
  S.phase = PH_TRIAL;
  if (P.restart == RAPDB_RESTART_FIXED && S.k == P.restart_period) {
    if (P.restart_from_average) {
      S.avg_pending = 1;
    } else {
      restart_scalars(P, S);
      S.restart_note = 1;
      if (quantised_refining(I, S)) S.phase = PH_KKT32;
    }
  }
}

__device__ void reject_trial(const Inst& I, State& S, Ctrl* ctrl) {
  S.trial += 1;
  if (S.trial >= I.P.max_trials) {
    finish(S, ctrl, RAPDB_ERR_BACKTRACK);
    return;
  }
  S.tau *= I.P.eta;
  S.phase = PH_TRIAL;
}

// ---------------------------------------------------------------------------
// k_vec: trial step / KKT partials / xy second sweep / averaged restart point
// ---------------------------------------------------------------------------
template <int ST>
__global__ void __launch_bounds__(NT) k_vec(const Inst* __restrict__ insts, State* __restrict__ states,
                                            Ctrl* __restrict__ ctrl, const int* __restrict__ vmap,
                                            float* __restrict__ XS, float* __restrict__ VS) {
  extern __shared__ double sm[];            // ys[m], yts[m]
  __shared__ double red[NWARP * NVP];
  __shared__ double vfin[NVP];
  const int b = vmap[blockIdx.x];
  const Inst& I = insts[b];
  State& S = states[b];
  const int phase = S.phase;
  if (!vec_phase(phase)) return;
  const DevParams& P = I.P;
  const int m = I.m, n = I.n, ldv = I.ldv;
  const int cb = blockIdx.x - I.vblk0;
  const int tid = threadIdx.x;
  const int fresh = S.fresh;
  const int k = S.k, it = S.it;
  double* ys = sm;
  double* yts = sm + m;

  const double tau = S.tau;
  const double sigma = S.gamma * tau;
  const double theta = S.sigma_prev / sigma;
  const double* ycur = I.yb[S.ycur];
  const double* gk = I.gb[S.gcur];
  const double* gp = (k == 0) ? gk : I.gb[S.gcur ^ 1];
  for (int i = tid; i < m; i += NT) {
    ys[i] = ycur[i];
    if (phase == PH_TRIAL && P.variant == RAPDB_YX) {
      const double s = (1.0 + theta) * gk[i] - theta * gp[i];
      yts[i] = fmax(0.0, ycur[i] + sigma * s);
    } else if (phase == PH_XY2) {
      yts[i] = I.yb[S.ycur ^ 1][i];
    } else {
      yts[i] = ycur[i];
    }
  }
  __syncthreads();
  if (cb == 0 && phase == PH_TRIAL && P.variant == RAPDB_YX)
    for (int i = tid; i < m; i += NT) I.yb[S.ycur ^ 1][i] = yts[i];

  const bool kkt_due = (phase == PH_TRIAL && fresh &&
                        ((P.kkt_every > 0 && it % P.kkt_every == 0) || it >= P.max_iter)) ||
                       phase == PH_KKT32B;
  const float* xk = I.xb[S.xcur];
  float* xt_out = I.xb[S.xcur ^ 1];
  const float* Uc = I.U[S.ucur];
  float* Un = I.U[S.ucur ^ 1];
  const float* c = I.c;
  double acc[NVP];
#pragma unroll
  for (int q = 0; q < NVP; ++q) acc[q] = 0.0;

  const int j = cb * NT + tid;
  if (j < n) {
    const double xj = (double)xk[j];
    const float xj32 = xk[j];
    const double c0 = c[j];
    const double q0d = (I.q0_kind == RAPDB_Q0_DIAG) ? (double)I.q0diag[j] : 0.0;
    if (phase == PH_TRIAL || phase == PH_KKT32B) {
      // U (or the float32 KKT pass output) at x^k
      const float* Us = (phase == PH_KKT32B) ? Un : Uc;
      const double u0 = (I.s_off ? q0d * (double)xj32 : (double)Us[j]);
      const double gf = u0 + c0;
      double gc = 0.0, gt = 0.0;
      for (int i = 1; i <= m; ++i) {
        const double v = (double)Us[(size_t)i * ldv + j] + (double)c[(size_t)i * ldv + j];
        gc += ys[i - 1] * v;
        gt += yts[i - 1] * v;
      }
      const double grad = gf + gc;
      if (kkt_due) {
        const double lo = I.lb[j], hi = I.ub[j];
        const double rs = (xj <= lo) ? fmax(-grad, 0.0) : ((xj >= hi) ? fmax(grad, 0.0) : fabs(grad));
        acc[V_RS] = rs * rs;
        acc[V_GF] = gf * gf;
        acc[V_GC] = gc * gc;
      }
      if (phase == PH_KKT32B) {
        if (I.s_off) Un[j] = (float)(q0d * (double)xj32);
      } else {
        // trial point
        double step;
        if (P.variant == RAPDB_YX) {
          step = gf + gt;
        } else {
          I.gx[S.gxcur][j] = grad;
          const double gprev = (k == 0) ? grad : I.gx[S.gxcur ^ 1][j];
          step = (1.0 + theta) * grad - theta * gprev;
        }
        const double lo = I.lb[j], hi = I.ub[j];
        const double xt = fmin(fmax(xj - tau * step, lo), hi);
        const float xt32 = (float)xt;
        const float d32 = xt32 - xj32;
        xt_out[j] = xt32;
        I.dv[j] = d32;
        acc[V_DD] = (double)d32 * (double)d32;
        if (I.s_off) {
          const float u0n = (float)(q0d * (double)xt32);
          const float w0 = (float)(q0d * (double)d32);
          Un[j] = u0n;
          I.W[j] = w0;
          acc[V_XU0] = (double)xt32 * (double)u0n;
          acc[V_DW0] = (double)d32 * (double)w0;
          acc[V_DU0] = (double)d32 * u0;
        }
        acc[V_CX0] = c0 * (double)xt32;
        acc[V_CD0] = c0 * (double)d32;
        if (ST == RAPDB_FP8) {
          for (int s = 0; s < I.M; ++s) {
            const float sc = I.qscale[(size_t)s * ldv + j];
            XS[(size_t)s * ldv + j] = sc * xt32;
            VS[(size_t)s * ldv + j] = sc * d32;
          }
        }
        if (fresh) {
          if (P.log_cap > 0 && it >= 1 && it <= P.log_cap && P.x_log)
            P.x_log[(size_t)(it - 1) * n + j] = xj32;
          if (P.restart_from_average && k >= 1)
            I.xcum[j] = (k == 1 ? 0.0 : I.xcum[j]) + S.t_last * xj;
        }
      }
    } else if (phase == PH_XY2) {
      // a = sum_i dy_i (u~_i + c_i),  b = Q(y^k) d = w_0 + sum_i y_i w_i
      const float* Ut = Un;
      double a = 0.0, bb = (double)I.W[j];
      for (int i = 1; i <= m; ++i) {
        const double dy = yts[i - 1] - ys[i - 1];
        a += dy * ((double)Ut[(size_t)i * ldv + j] + (double)c[(size_t)i * ldv + j]);
        bb += ys[i - 1] * (double)I.W[(size_t)i * ldv + j];
      }
      acc[V_AA] = a * a;
      acc[V_BB] = bb * bb;
    } else if (phase == PH_INIT || phase == PH_AVG) {
      // the new start point: x^0 itself, or the weighted average of the run
      const float xt32 = (phase == PH_INIT) ? xj32 : (float)(I.xcum[j] / S.T);
      xt_out[j] = xt32;
      I.dv[j] = 0.0f;
      if (I.s_off) {
        const float u0n = (float)(q0d * (double)xt32);
        Un[j] = u0n;
        I.W[j] = 0.0f;
        acc[V_XU0] = (double)xt32 * (double)u0n;
      }
      acc[V_CX0] = c0 * (double)xt32;
      if (ST == RAPDB_FP8) {
        for (int s = 0; s < I.M; ++s) {
          XS[(size_t)s * ldv + j] = I.qscale[(size_t)s * ldv + j] * xt32;
          VS[(size_t)s * ldv + j] = 0.0f;
        }
      }
    }
  }
  if (cb == 0 && tid == 0 && fresh && phase == PH_TRIAL && P.log_cap > 0 && it >= 1 && it <= P.log_cap &&
      P.y_log) {
    for (int i = 0; i < m; ++i) P.y_log[(size_t)(it - 1) * m + i] = (float)ys[i];
  }

  block_sum<NVP>(acc, red);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NVP; ++q) I.vpart[(size_t)cb * NVP + q] = acc[q];
  }
  if (!arrive_last(&S.arrive_vec, (unsigned)I.ncb)) return;

  // ---- last CTA of this instance: fixed-order reduction + control ----
  if (tid < NVP) {
    double s = 0.0;
    for (int bq = 0; bq < I.ncb; ++bq) s += __ldcg(&I.vpart[(size_t)bq * NVP + tid]);
    vfin[tid] = s;
  }
  __syncthreads();
  if (tid != 0) return;

  if (phase == PH_INIT || phase == PH_AVG || phase == PH_TRIAL) {
    S.dd = vfin[V_DD];
    for (int q = 0; q < NDOT; ++q) S.dots0[q] = vfin[V_XU0 + q];
  }
  if (phase == PH_TRIAL && fresh) {
    if (kkt_due) {
      double rel, rs, rf;
      kkt_from_partials(I, gk, ys, vfin[V_RS], vfin[V_GF], vfin[V_GC], rel, rs, rf);
      S.rel_kkt = rel;
      S.r_stat = rs;
      S.r_feas = rf;
      if (!(rel == rel)) { finish(S, ctrl, RAPDB_ERR_NUMERIC); return; }
      if (quantised_refining(I, S)) {
        S.rel_q = rel;
        if (rel <= P.tol) { S.phase = PH_KKT32; return; }
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
    if (P.restart == RAPDB_RESTART_GAP && it >= P.gap_first &&
        (it == P.gap_first || (it - P.gap_first) % P.gap_every == 0) && S.gap_iter == 0) {
      // smoothed-gap evaluation at this iterate before the iteration
      S.fresh = 0;
      S.gap_iter = 1;
      S.phase = PH_GAPY;
      return;
    }
    S.restarts += S.restart_note;
    S.restart_note = 0;
    S.fresh = 0;
    return;
  }
  if (phase == PH_XY2) {
    const double tau_ = S.tau;
    const double sig = S.gamma * tau_;
    const double th = S.sigma_prev / sig;
    double ddy = 0.0;
    for (int i = 0; i < m; ++i) { const double t = yts[i] - ys[i]; ddy += t * t; }
    ddy *= 0.5;
    const double dp = 0.5 * S.dd;
    const double an = P.c_alpha / tau_;
    const double bn = P.gamma0 * P.c_beta / sig;
    const double bterm = (bn > 0.0) ? vfin[V_BB] / (2.0 * bn) : (vfin[V_BB] == 0.0 ? 0.0 : INFINITY);
    const double E = vfin[V_AA] / (2.0 * an) - ddy / sig + bterm - (1.0 / tau_ - th * (S.alpha_k + S.beta_k)) * dp;
    const bool ok = E <= -P.delta / tau_ * dp - P.delta / sig * ddy;
    S.trials_total += 1;
    if (!(E == E)) { finish(S, ctrl, RAPDB_ERR_NUMERIC); return; }
    if (ok || !P.backtracking) accept_trial(I, S, sig, an, bn);
    else reject_trial(I, S, ctrl);
    return;
  }
  if (phase == PH_KKT32B) {
    double rel, rs, rf;
    kkt_from_partials(I, I.gnew, ys, vfin[V_RS], vfin[V_GF], vfin[V_GC], rel, rs, rf);
    S.rel_kkt = rel;
    S.r_stat = rs;
    S.r_feas = rf;
    if (rel <= P.tol) { finish(S, ctrl, RAPDB_OK); return; }
    const bool stalled = (S.kkt_ref > 0.0 && rel > P.stall_ratio * S.kkt_ref);
    S.kkt_ref = rel;
    if (stalled || S.rel_q <= P.tol) {
      // switch to the float32 Q: the KKT pass output becomes the current U
      S.precision = 1;
      S.switches += 1;
      S.ucur ^= 1;
      double* gd = I.gb[S.gcur];
      for (int i = 0; i < m; ++i) gd[i] = I.gnew[i];
      restart_scalars(P, S);
      S.restart_note = 1;
    }
    S.fresh = 1;
    S.phase = PH_TRIAL;
    return;
  }
}

// ---------------------------------------------------------------------------
// k_pass: the fused coupling pass + post-control
// ---------------------------------------------------------------------------
template <int ST>
__global__ void __launch_bounds__(NT) k_pass(const Inst* __restrict__ insts, State* __restrict__ states,
                                             Ctrl* __restrict__ ctrl, const int* __restrict__ pmap,
                                             const float* __restrict__ XS, const float* __restrict__ VS) {
  __shared__ double red[NWARP * NDOT];
  const int b = pmap[blockIdx.x];
  const Inst& I = insts[b];
  State& S = states[b];
  const int phase = S.phase;
  if (!pass_phase(phase)) return;
  const int item = blockIdx.x - I.pblk0;
  const int s = item / I.nrb;
  const int r = item - s * I.nrb;
  const int i = s + I.s_off;
  const int row0 = r * I.rb;
  const int rows = min(I.rb, I.n - row0);
  const int ldv = I.ldv;
  const bool use32 = (phase == PH_KKT32) || (ST != RAPDB_F32 && S.precision == 1);
  const float* x = (phase == PH_KKT32) ? I.xb[S.xcur] : I.xb[S.xcur ^ 1];
  const float* v = (phase == PH_KKT32) ? I.xb[S.xcur] : I.dv;
  const float* uold = (phase == PH_KKT32) ? nullptr : I.U[S.ucur] + (size_t)i * ldv;
  float* Uo = I.U[S.ucur ^ 1] + (size_t)i * ldv;
  float* Wo = I.W + (size_t)i * ldv;
  double* out = I.part + (size_t)s * NDOT * I.nrb + r;
  const float* crow = I.c + (size_t)i * ldv;
  if (use32 || ST == RAPDB_F32) {
    const float* Qb = (ST == RAPDB_F32 && !use32) ? (const float*)I.Q : I.Q32;
    const int ldq = (ST == RAPDB_F32 && !use32) ? I.ld : I.ld32;
    pass_block<RAPDB_F32, 4, 2>((const uint8_t*)(Qb + (size_t)s * I.n * ldq), ldq, row0, rows, x, v, nullptr,
                                nullptr, nullptr, uold, crow, Uo, Wo, out, I.nrb, red);
  } else {
    constexpr int EB = Elt<ST>::B;
    const uint8_t* Qb = (const uint8_t*)I.Q + (size_t)s * I.n * I.ld * EB;
    pass_block<ST, 4, 2>(Qb, I.ld, row0, rows, x, v, XS ? XS + (size_t)s * ldv : nullptr,
                         VS ? VS + (size_t)s * ldv : nullptr, I.qscale ? I.qscale + (size_t)s * ldv : nullptr,
                         uold, crow, Uo, Wo, out, I.nrb, red);
  }
  if (!arrive_last(&S.arrive_pass, (unsigned)(I.M * I.nrb))) return;

  // ---- last CTA: fixed-order reduction of the block partials ----
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pq = warp; pq < I.M * NDOT; pq += NWARP) {
    const double* src = I.part + (size_t)pq * I.nrb;
    double t = 0.0;
    for (int rr = lane; rr < I.nrb; rr += 32) t += __ldcg(src + rr);
    t = warp_sum(t);
    if (lane == 0) {
      const int ss = pq / NDOT, q = pq - ss * NDOT;
      I.dots[(size_t)(ss + I.s_off) * NDOT + q] = t;
    }
  }
  if (I.s_off && threadIdx.x < NDOT) I.dots[threadIdx.x] = S.dots0[threadIdx.x];
  __threadfence_block();
  __syncthreads();
  if (threadIdx.x != 0) return;

  const DevParams& P = I.P;
  const int m = I.m;
  const double* D = I.dots;
  S.passes += 1;
  // g at the pass point: g_i = 0.5 x'Q_i x + c_i'x + d_i
  for (int ii = 1; ii <= m; ++ii)
    I.gnew[ii - 1] = 0.5 * __ldcg(&D[ii * NDOT + D_XU]) + __ldcg(&D[ii * NDOT + D_CX]) + I.dcon[ii - 1];

  if (phase == PH_INIT || phase == PH_AVG) {
    S.xcur ^= 1;
    S.ucur ^= 1;
    double* gd = I.gb[S.gcur];
    for (int ii = 0; ii < m; ++ii) gd[ii] = I.gnew[ii];
    S.obj = 0.5 * D[D_XU] + D[D_CX];
    if (phase == PH_INIT) {
      S.fresh = 1;
      S.phase = PH_TRIAL;
    } else {
      double* y = I.yb[S.ycur];
      for (int ii = 0; ii < m; ++ii) y[ii] = I.ycum[ii] / S.T;
      restart_scalars(P, S);
      S.restarts += 1;
      S.fresh = 0;       // the KKT test of this iteration ran at the last iterate
      S.phase = PH_TRIAL;
    }
    return;
  }
  if (phase == PH_KKT32) {
    S.phase = PH_KKT32B;
    return;
  }
  if (phase == PH_TRIAL) {
    const double tau = S.tau;
    const double sig = S.gamma * tau;
    const double th = S.sigma_prev / sig;
    if (P.variant == RAPDB_YX) {
      const double* yt = I.yb[S.ycur ^ 1];
      const double* y = I.yb[S.ycur];
      double dQd = D[D_VW], dg2 = 0.0, dy2 = 0.0;
      for (int ii = 1; ii <= m; ++ii) {
        const double vw = D[ii * NDOT + D_VW];
        dQd += yt[ii - 1] * vw;
        const double dgi = D[ii * NDOT + D_VUO] + D[ii * NDOT + D_CV] + 0.5 * vw;
        dg2 += dgi * dgi;
        const double t = yt[ii - 1] - y[ii - 1];
        dy2 += t * t;
      }
      const double an = P.c_alpha / sig;
      const double E = 0.5 * dQd - S.dd / (2.0 * tau) + dg2 / (2.0 * an) -
                       (1.0 / sig - th * S.alpha_k) * 0.5 * dy2;
      const bool ok = E <= -P.delta * S.dd / (2.0 * tau) - P.delta * dy2 / (2.0 * sig);
      S.trials_total += 1;
      if (!(E == E)) { finish(S, ctrl, RAPDB_ERR_NUMERIC); return; }
      if (ok || !P.backtracking) accept_trial(I, S, sig, an, 0.0);
      else reject_trial(I, S, ctrl);
    } else {
      // xy: dual ascent at the new primal point, then the a/b sweep
      const double* y = I.yb[S.ycur];
      double* yt = I.yb[S.ycur ^ 1];
      for (int ii = 0; ii < m; ++ii) yt[ii] = fmax(0.0, y[ii] + sig * I.gnew[ii]);
      (void)th;
      S.phase = PH_XY2;
    }
    return;
  }
}

}  // namespace rapdb_dev
