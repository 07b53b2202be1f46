// Set-up and stand-alone kernels: storage conversion (BF16 / Jacobi-scaled
// FP8), input validation, state initialisation, the stand-alone coupling pass
// and KKT residual used by rapdb_coupling_pass / rapdb_kkt_residual.
#pragma once
#include "rapdb_kernels.cuh"

namespace rapdb_dev {

// ---- storage conversion (one pass over Q) --------------------------------
// BF16: round to nearest, ties to even.
__global__ void k_quant_bf16(const float* __restrict__ Q, int n, long long rows, int ld,
                             __nv_bfloat16* __restrict__ out) {
  const long long total = rows * (long long)n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n;
    const int col = (int)(e - r * n);
    out[r * ld + col] = __float2bfloat16_rn(Q[e]);
  }
}

// FP8 symmetric Jacobi scaling: r_j = 1/sqrt(Q_jj) (1 when Q_jj <= 0),
// C_jk = (Q_jk (r_j r_k)) 256 rounded to E4M3 (nearest even, saturating),
// s_j = sqrt(Q_jj)/16 (1/16 when Q_jj <= 0), so Q~ = S dec(C) S.  The factor
// r_j r_k is formed first, so C (and Q~) is exactly symmetric, which the
// packed upper block triangle relies on.
__global__ void k_fp8_scales(const float* __restrict__ Q, int n, int M, int ldv, float* __restrict__ rinv,
                             float* __restrict__ scale) {
  const long long total = (long long)M * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n);
    const int j = (int)(e - (long long)s * n);
    const float dg = Q[((size_t)s * n + j) * n + j];
    const float sq = dg > 0.0f ? __fsqrt_rn(dg) : 1.0f;
    rinv[(size_t)s * ldv + j] = __fdiv_rn(1.0f, sq);
    scale[(size_t)s * ldv + j] = sq * (1.0f / 16.0f);
  }
}

__global__ void k_quant_fp8(const float* __restrict__ Q, int n, int M, int ld, int ldv,
                            const float* __restrict__ rinv, __nv_fp8_storage_t* __restrict__ out) {
  const long long total = (long long)M * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n;          // global row (s * n + j)
    const int col = (int)(e - r * n);
    const int s = (int)(r / n);
    const int j = (int)(r - (long long)s * n);
    const float rr = __fmul_rn(rinv[(size_t)s * ldv + j], rinv[(size_t)s * ldv + col]);
    const float cval = __fmul_rn(__fmul_rn(Q[e], rr), 256.0f);
    out[r * ld + col] = __nv_cvt_float_to_fp8(cval, __NV_SATFINITE, __NV_E4M3);
  }
}

// ---- symmetric block packing ------------------------------------------------
// flag = 1 when some Q_s[j][k] != Q_s[k][j]: 32 x 32 blocks (bi, bj), bi <= bj,
// the mirror block staged through shared memory so both reads coalesce.
__global__ void k_sym_check(const float* __restrict__ Q, int ld, int n, int M, int* flag) {
  __shared__ float a[32][33];
  const int nb = (n + 31) / 32;
  const int64_t total = (int64_t)M * nb * nb;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int s = (int)(b / ((int64_t)nb * nb));
    const int rem = (int)(b - (int64_t)s * nb * nb);
    const int bi = rem / nb, bj = rem - bi * nb;
    if (bi > bj) continue;     // uniform over the CTA
    const float* Qs = Q + (size_t)s * n * ld;
    for (int r = ty; r < 32; r += 8) {
      const int row = bj * 32 + r, col = bi * 32 + tx;
      a[r][tx] = (row < n && col < n) ? Qs[(size_t)row * ld + col] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int row = bi * 32 + r, col = bj * 32 + tx;
      if (row < n && col < n && Qs[(size_t)row * ld + col] != a[tx][r]) atomicOr(flag, 1);
    }
    __syncthreads();
  }
}

// Qp[s][t] = Q_s[I*STB .. , J*STB .. ] for tile t = (I, J) of tij, zero
// outside n x n.
__global__ void k_pack_sym(const float* __restrict__ Q, int ld, int n, int M, int T, int ntile,
                           const int* __restrict__ tij, float* __restrict__ Qp) {
  const int64_t total = (int64_t)M * ntile * STB * STB;
  (void)T;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % STB);
    const int r = (int)((e / STB) % STB);
    const int64_t st = e / ((int64_t)STB * STB);
    const int t = (int)(st % ntile);
    const int s = (int)(st / ntile);
    const int ij = tij[t];
    const int row = (ij >> 16) * STB + r, col = (ij & 0xffff) * STB + c;
    Qp[e] = (row < n && col < n) ? Q[(size_t)s * n * ld + (size_t)row * ld + col] : 0.f;
  }
}

// The same tiles of the quantised stored matrices (EB-byte codes, row
// stride ld): Qp[s][t] = codes of Q~_s[I*STB .., J*STB ..], zero outside n x n
// (a zero code is 0.0 in BF16 and in E4M3), in the tensor cores' core-matrix
// layout: entry (r, c) of a tile at ((r / 8) NC + c / CE) 128 B + (r % 8) 16 B +
// (c % CE) EB, CE = 16 / EB entries per 16-byte core row, NC = STB / CE.
template <typename T_>
__global__ void k_pack_sym_codes(const T_* __restrict__ Q, int ld, int n, int M, int ntile,
                                 const int* __restrict__ tij, T_* __restrict__ Qp) {
  constexpr int CE = 16 / (int)sizeof(T_), NC = STB / CE, PER_CORE = 128 / (int)sizeof(T_);
  const int64_t total = (int64_t)M * ntile * STB * STB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % STB);
    const int r = (int)((e / STB) % STB);
    const int64_t st = e / ((int64_t)STB * STB);
    const int t = (int)(st % ntile);
    const int s = (int)(st / ntile);
    const int ij = tij[t];
    const int row = (ij >> 16) * STB + r, col = (ij & 0xffff) * STB + c;
    const int64_t dst = st * STB * STB + (int64_t)((r >> 3) * NC + c / CE) * PER_CORE + (r & 7) * CE + (c % CE);
    Qp[dst] = (row < n && col < n) ? Q[(size_t)s * n * ld + (size_t)row * ld + col] : T_(0);
  }
}

// dots[(s + s_off) * NDOT + q] = sum over the T row blocks of spart[s][q][.]
// (the same row-block order and double-float sums as the solver's control
// kernel).
__global__ void __launch_bounds__(NT) k_sym_dots(const Inst* __restrict__ insts, const float2* __restrict__ spart,
                                                double* __restrict__ dots) {
  const Inst& I = insts[0];
  const int T = I.tsym;
  for (int pq = threadIdx.x; pq < I.M * NDOT; pq += NT) {
    const int ss = pq / NDOT, q = pq - ss * NDOT;
    dots[(size_t)(ss + I.s_off) * NDOT + q] = df_to_double(df_sum_pairs(spart + (size_t)pq * T, T));
  }
}

// ---- validation: NaN / Inf anywhere, negative diagonal, lb > ub ----------
__global__ void k_validate(const float* __restrict__ Q, int n, int M, const float* __restrict__ c, int m,
                           const float* __restrict__ d, const float* __restrict__ lb,
                           const float* __restrict__ ub, const float* __restrict__ q0diag,
                           int* __restrict__ flags) {
  const long long totalQ = (long long)M * n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int bad_nan = 0, bad_diag = 0, bad_box = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totalQ; e += stride) {
    const float v = Q[e];
    if (!isfinite(v)) bad_nan = 1;
    const long long r = e / n;
    const int col = (int)(e - r * n);
    if ((int)(r % n) == col && v < 0.0f) bad_diag = 1;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)(m + 1) * n; e += stride)
    if (!isfinite(c[e])) bad_nan = 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += stride) {
    // bounds may be infinite (lb = -inf, ub = +inf), not NaN
    if (isnan(lb[e]) || isnan(ub[e])) bad_nan = 1;
    if (lb[e] > ub[e] || lb[e] == INFINITY || ub[e] == -INFINITY) bad_box = 1;
    if (q0diag) {
      if (!isfinite(q0diag[e])) bad_nan = 1;
      if (q0diag[e] < 0.0f) bad_diag = 1;
    }
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += stride)
    if (!isfinite(d[e])) bad_nan = 1;
  if (bad_nan) atomicOr(&flags[0], 1);
  if (bad_diag) atomicOr(&flags[1], 1);
  if (bad_box) atomicOr(&flags[2], 1);
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int len) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) b[e] = (double)a[e];
}
__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int len) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) b[e] = (float)a[e];
}

// Start-of-solve state: x^0 into slot 0 (checked against the box), y^0 into
// slot 0 (checked >= 0), Algorithm 1's initial scalars, deadline.
__global__ void __launch_bounds__(NT) k_init_state(Inst* __restrict__ insts, State* __restrict__ states, int B,
                                                   double time_limit_s, int* __restrict__ flags) {
  __shared__ double red[NWARP];
  const int b = blockIdx.x;
  if (b >= B) return;
  const Inst& I = insts[b];
  double ax[1] = {0.0}, axa[1] = {0.0};
  for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
    const float x = I.xf[0][j];
    I.xb[0][j] = (double)x;
    I.xl[0][j] = 0.0f;
    if (!(x >= I.lb[j] && x <= I.ub[j])) atomicOr(&flags[0], 1);
    if (I.hyp_a) {
      ax[0] += (double)I.hyp_a[j] * (double)x;
      axa[0] += fabs((double)I.hyp_a[j] * (double)x);
    }
  }
  if (I.hyp_a) {
    // x0 must lie on the hyperplane of X (to the float32 rounding of its data)
    block_allsum<1>(ax, red);
    block_allsum<1>(axa, red);
    if (threadIdx.x == 0 && !(fabs(ax[0] - I.hyp_beta) <= 1e-6 * (1.0 + axa[0] + fabs(I.hyp_beta))))
      atomicOr(&flags[0], 2);
  }
  for (int i = threadIdx.x; i < I.m; i += blockDim.x)
    if (i < I.m_ineq ? !(I.yb[0][i] >= 0.0) : !(fabs(I.yb[0][i]) < INFINITY)) atomicOr(&flags[1], 1);
  if (threadIdx.x != 0) return;
  if (I.P.dual_simplex && I.m_ineq > 0) {
    // a simplex dual start must lie on the simplex
    double sy = 0.0;
    for (int i = 0; i < I.m_ineq; ++i) sy += I.yb[0][i];
    if (!(fabs(sy - I.P.dual_r) <= 1e-6 * I.P.dual_r)) atomicOr(&flags[1], 2);
  }
  State& S = states[b];
  const unsigned long long now = globaltimer();
  S = State{};
  restart_scalars(I.P, S);
  S.sigma0 = S.sigma_prev;
  S.phase = PH_INIT;
  // float32 storage with refinement runs the compensated level from the
  // start; quantised storage with packed tiles its quantised-increment level
  if (I.P.refine && I.storage == RAPDB_F32 && I.Ulo[0]) S.precision = 2;
  else if (I.P.refine && I.Qpq && I.Ulo[0]) S.precision = 3;
  S.switch_it = -1;
  S.rel_kkt = S.r_stat = S.r_feas = NAN;
  S.rel_q = INFINITY;
  S.gap_it_done = -1;
  S.deadline_ns = time_limit_s > 0.0 ? (long long)(now + (unsigned long long)(time_limit_s * 1e9)) : 0;
}

// Q_0 row of a stand-alone pass when Q_0 is diagonal or zero, plus the FP8
// pre-scaled right-hand sides; per-block partials of the i = 0 dots.
__global__ void __launch_bounds__(NT) k_vec_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                  const float* __restrict__ v, const float* __restrict__ uold,
                                                  float* __restrict__ U, float* __restrict__ W,
                                                  float* __restrict__ XS, float* __restrict__ VS,
                                                  double* __restrict__ vpart, int use32) {
  __shared__ double red[NWARP * NDOT];
  const Inst& I = insts[0];
  const int j = blockIdx.x * NT + threadIdx.x;
  double acc[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (j < I.n) {
    const float xj = x[j], vj = v[j];
    if (I.storage == RAPDB_FP8 && !use32) {
      for (int s = 0; s < I.M; ++s) {
        const float sc = I.qscale[(size_t)s * I.ldv + j];
        XS[(size_t)s * I.ldv + j] = sc * xj;
        VS[(size_t)s * I.ldv + j] = sc * vj;
      }
    }
    if (I.s_off) {
      const double q0d = (I.q0_kind == RAPDB_Q0_DIAG) ? (double)I.q0diag[j] : 0.0;
      const float u = (float)(q0d * xj), w = (float)(q0d * vj);
      U[j] = u;
      W[j] = w;
      acc[D_XU] = (double)xj * u;
      acc[D_VW] = (double)vj * w;
      acc[D_VUO] = uold ? (double)vj * uold[j] : 0.0;
      acc[D_CX] = (double)I.c[j] * xj;
      acc[D_CV] = (double)I.c[j] * vj;
    }
  }
  block_sum<NDOT>(acc, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < NDOT; ++q) vpart[(size_t)blockIdx.x * NDOT + q] = acc[q];
}

// Fixed-order final reduction of a stand-alone pass into dots[(m+1)][5].
__global__ void __launch_bounds__(NT) k_dots_final(const Inst* __restrict__ insts, const double* __restrict__ part,
                                                   const double* __restrict__ vpart, double* __restrict__ dots,
                                                   const float* __restrict__ x, const float* __restrict__ v) {
  __shared__ double red[NWARP * 2];
  const Inst& I = insts[0];
  // linear equalities (no stored matrix): u = w = 0, c'x and c'v
  for (int i = I.m_ineq + 1; i <= I.m; ++i) {
    const float* ci = I.c + (size_t)i * I.ldv;
    double sv[2] = {0.0, 0.0};
    for (int jj = threadIdx.x; jj < I.n; jj += NT) {
      sv[0] += (double)ci[jj] * (double)x[jj];
      sv[1] += (double)ci[jj] * (double)v[jj];
    }
    block_allsum<2>(sv, red);
    if (threadIdx.x == 0) {
      double* Di = dots + (size_t)i * NDOT;
      Di[D_XU] = 0.0;
      Di[D_VW] = 0.0;
      Di[D_VUO] = 0.0;
      Di[D_CX] = sv[0];
      Di[D_CV] = sv[1];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pq = warp; pq < I.M * NDOT; pq += NWARP) {
    const double* src = part + (size_t)pq * I.nrb;
    double t = 0.0;
    for (int rr = lane; rr < I.nrb; rr += 32) t += src[rr];
    t = warp_sum(t);
    if (lane == 0) {
      const int ss = pq / NDOT, q = pq - ss * NDOT;
      dots[(size_t)(ss + I.s_off) * NDOT + q] = t;
    }
  }
  if (I.s_off && threadIdx.x < NDOT) {
    double t = 0.0;
    for (int bq = 0; bq < I.ncb; ++bq) t += vpart[(size_t)bq * NDOT + threadIdx.x];
    dots[threadIdx.x] = t;
  }
}

// KKT partials at (x, y) from U = Q x (row 0 from the diagonal when Q_0 is
// not stored): ||r_stat||^2, ||Q_0x+c_0||^2, ||sum_i y_i(Q_ix+c_i)||^2.
__global__ void __launch_bounds__(NT) k_kkt_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                  const double* __restrict__ y, const float* __restrict__ U,
                                                  const float* __restrict__ Ulo, double* __restrict__ vpart) {
  __shared__ double red[NWARP * 3];
  const Inst& I = insts[0];
  const int j = blockIdx.x * NT + threadIdx.x;
  double acc[3] = {0.0, 0.0, 0.0};
  if (j < I.n) {
    const double xj = x[j];
    const double u0 = I.s_off ? ((I.q0_kind == RAPDB_Q0_DIAG) ? (double)I.q0diag[j] * (double)x[j] : 0.0)
                              : (double)U[j] + (Ulo ? (double)Ulo[j] : 0.0);
    const double gf = u0 + (double)I.c[j];
    double gc = 0.0;
    for (int i = 1; i <= I.m; ++i)
      gc += y[i - 1] * ((double)U[(size_t)i * I.ldv + j] + (Ulo ? (double)Ulo[(size_t)i * I.ldv + j] : 0.0) +
                        (double)I.c[(size_t)i * I.ldv + j]);
    const double grad = gf + gc;
    if (I.hyp_a) {   // dist(0, grad + N_X(x)) needs every column: formed in k_kkt_final
      const dflt gd = df_from_double(grad);
      I.hg[j] = make_float2(gd.hi, gd.lo);
    } else {
      const double lo = I.lb[j], hi = I.ub[j];
      const double rs = (xj <= lo) ? fmax(-grad, 0.0) : ((xj >= hi) ? fmax(grad, 0.0) : fabs(grad));
      acc[0] = rs * rs;
    }
    acc[1] = gf * gf;
    acc[2] = gc * gc;
  }
  block_sum<3>(acc, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) vpart[(size_t)blockIdx.x * 3 + q] = acc[q];
}

// (one CTA of NT threads; x, xlo: the point as a float pair, for the
// hyperplane's cone residual)
__global__ void __launch_bounds__(NT) k_kkt_final(const Inst* __restrict__ insts, const double* __restrict__ vpart,
                                                  const double* __restrict__ dots, const double* __restrict__ y,
                                                  double* __restrict__ g, double* __restrict__ out,
                                                  const float* __restrict__ x, const float* __restrict__ xlo) {
  __shared__ float2 hsm[NWARP + 2];
  __shared__ double hsb[2];
  const Inst& I = insts[0];
  double rs2h = 0.0;
  if (I.hyp_a) rs2h = hyp_cone_rs2(I, x, xlo, 0.0, nullptr, hsm, hsb);
  if (threadIdx.x != 0) return;
  double p[3] = {0.0, 0.0, 0.0};
  for (int bq = 0; bq < I.ncb; ++bq)
    for (int q = 0; q < 3; ++q) p[q] += vpart[(size_t)bq * 3 + q];
  if (I.hyp_a) p[0] = rs2h;
  for (int i = 1; i <= I.m; ++i) g[i - 1] = 0.5 * dots[i * NDOT + D_XU] + dots[i * NDOT + D_CX] + I.dcon[i - 1];
  double rf2 = 0.0, gd2 = 0.0;
  const double tc = I.P.dual_simplex ? simplex_cone_t_serial(g, y, I.m_ineq) : 0.0;
  for (int i = 0; i < I.m; ++i) {
    double ri;
    if (i >= I.m_ineq) ri = g[i];               // equality: |a'x - b|
    else if (I.P.dual_simplex) ri = (y[i] > 0.0) ? g[i] - tc : fmax(g[i] - tc, 0.0);
    else ri = (y[i] > 0.0) ? fabs(g[i]) : fmax(g[i], 0.0);
    rf2 += ri * ri;
    const double t = g[i] - I.dcon[i];
    gd2 += t * t;
  }
  double rel, rs, rf;
  kkt_finish(I, p[0], p[1], p[2], rf2, gd2, rel, rs, rf);
  out[0] = rel;
  out[1] = rs;
  out[2] = rf;
  out[3] = 0.5 * dots[D_XU] + dots[D_CX];
}

}  // namespace rapdb_dev
