// Symmetric block packing of the coupling pass.
//
// Every Q_i of the problem class is symmetric, so its upper block triangle
// determines it.  The packed copy keeps the tiles (I, J), I <= J, of
// STB x STB entries (row-major inside a tile, zero outside n x n).  An
// off-diagonal tile B = Q_i[I, J] serves both B d_J (rows of block I) and
// B' d_I (rows of block J), so a pass reads each entry of Q_i once where the
// row-streaming pass reads the off-diagonal ones twice: half the bytes.
//
// The transposed products land in rows that other CTAs own.  Each tile
// product goes to its own slot of a partial buffer (slot J of the rows of
// block I); a second kernel, one CTA per row block, sums the block's T slots
// in slot order (a compensated float32 sum), then applies the incremental
// compensated update of the trial pass:
//   w = (Q_i d)_j,  u = U^k_j (double-float) + w,  U' = hi/lo of u,  W = w,
// with the per-row dots x'u, v'w, v'U^k, c'x, c'v.  The tile kernel streams
// with no counters or fences (the kernel boundary orders its stores before
// the reduction), and every sum has a fixed order: runs are bit-for-bit
// reproducible.
//
// The packed pass serves the incremental trials (U' = U^k + Q d at the
// compensated level, the dominant pass of a solve) and the smoothed gap's
// two-right-hand-side passes over the float32 matrices (U = Q x, W = Q v);
// the direct compensated anchors, the setup and check passes and the passes
// over quantised matrices keep the row-streaming tile.
#pragma once

namespace rapdb_dev {

constexpr int STB = 128;             // tile edge (rows of a row block)
static_assert(NT == 2 * STB, "the row-block reduction splits the T slots over two halves of the CTA");

// The passes the packed tiles serve: 1 = the incremental compensated trial
// pass (U' = U^k + Q d, one right-hand side), 2 = a smoothed-gap pass over
// the float32 matrices (U = Q x, W = Q v, plain float32 products, two
// right-hand sides); 0 = any other pass (the row-streaming tile runs it).
__device__ __forceinline__ int sym_kind(const Inst& I, const State& S) {
  if (I.tsym == 0) return 0;
  const int ph = S.phase;
  if (ph == PH_TRIAL) return (S.trial_ready && S.precision == 2 && S.anchor_age < ANCHOR_EVERY) ? 1 : 0;
  if (gap_phase(ph)) return (I.storage == RAPDB_F32 || S.precision >= 1) ? 2 : 0;
  return 0;
}

// Row block R of stored matrix s (constraint row i) is complete: sum its T
// slots in slot order, apply the incremental update and write the block's dot
// partials to out[q * T].  The slot sums are compensated float32 sums
// (Knuth's TwoSum per addition, the rounding errors summed alongside): within
// 2u of the exact sum plus O(T^2 u^2) of the sum of |slots|, with no float64
// work (float64 runs at a small fraction of the float32 rate on this GPU).
// The two halves of the CTA take half the slots each; the low half's sum
// absorbs the high half's with one more TwoSum.  The update and the five dots
// are float64; the dots are summed over the 128 rows through shared memory
// (four rows per lane, then a fixed warp tree).  xl, uol and Uol may be null
// (zero low parts, no low output).  `sh` = NDOT x STB doubles.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float a) {
  const float t = s + a;
  const float z = t - s;
  c += (s - (t - z)) + (a - z);
  s = t;
}

static __device__ void sym_rows(const Inst& I, const float* __restrict__ Ps, int R, int i,
                                const float* __restrict__ x, const float* __restrict__ xl,
                                const float* __restrict__ v, const float* __restrict__ uoh,
                                const float* __restrict__ uol, float* __restrict__ Uoh, float* __restrict__ Uol,
                                float* __restrict__ W, double* __restrict__ out, double* sh) {
  const int T = I.tsym;
  const size_t ldp = (size_t)T * STB;
  const int tid = threadIdx.x, t = tid & (STB - 1), half = tid / STB;
  const int h = T / 2;
  const int s0 = half ? h : 0, s1 = half ? T : h;
  const float* src = Ps + (size_t)R * STB + t;
  float sa = 0.f, ca = 0.f;
#pragma unroll 8
  for (int sl = s0; sl < s1; ++sl) two_sum_acc(sa, ca, __ldcg(src + (size_t)sl * ldp));
  float2* shf = reinterpret_cast<float2*>(sh);
  if (half) shf[t] = make_float2(sa, ca);
  __syncthreads();
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int j = R * STB + t;
  if (!half) {
    const float2 hi = shf[t];
    two_sum_acc(sa, ca, hi.x);
    ca += hi.y;
    if (j < I.n) {
      const double w = (double)sa + (double)ca;
      const size_t o = (size_t)i * I.ldv + j;
      const double uo = (double)uoh[o] + (uol ? (double)uol[o] : 0.0);
      const double u = uo + w;
      const float uh = (float)u;
      Uoh[o] = uh;
      if (Uol) Uol[o] = (float)(u - (double)uh);
      W[o] = (float)w;
      const double xj = (double)x[j] + (xl ? (double)xl[j] : 0.0), vj = v[j], cj = I.c[o];
      dsum[0] = xj * u;
      dsum[1] = vj * w;
      dsum[2] = vj * uo;
      dsum[3] = cj * xj;
      dsum[4] = cj * vj;
    }
  }
  __syncthreads();   // shf is read
  if (!half) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) sh[q * STB + t] = dsum[q];
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  if (warp < NDOT) {
    const double* r = sh + warp * STB;
    double a = r[lane];
#pragma unroll
    for (int k = 1; k < STB / 32; ++k) a += r[lane + 32 * k];
    a = warp_sum(a);
    if (lane == 0) out[(size_t)warp * T] = a;
  }
  __syncthreads();   // sh is reused by the caller
}

// The same for a two-right-hand-side pass (kind 2): U = Q_i x and W = Q_i v
// from the two slot sets Px, Pv (compensated float32 slot sums, one final
// rounding each), dots x'U, v'W, 0, c'x, c'v in float64 as the row-streaming
// pass forms them.
static __device__ void sym_rows2(const Inst& I, const float* __restrict__ Px, const float* __restrict__ Pv, int R,
                                 int i, const float* __restrict__ x, const float* __restrict__ v,
                                 float* __restrict__ U, float* __restrict__ W, double* __restrict__ out, double* sh) {
  const int T = I.tsym;
  const size_t ldp = (size_t)T * STB;
  const int tid = threadIdx.x, t = tid & (STB - 1), half = tid / STB;
  const int h = T / 2;
  const int s0 = half ? h : 0, s1 = half ? T : h;
  const size_t off = (size_t)R * STB + t;
  float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
#pragma unroll 4
  for (int sl = s0; sl < s1; ++sl) {
    two_sum_acc(sa, ca, __ldcg(Px + off + (size_t)sl * ldp));
    two_sum_acc(sb, cb, __ldcg(Pv + off + (size_t)sl * ldp));
  }
  float4* shf = reinterpret_cast<float4*>(sh);
  if (half) shf[t] = make_float4(sa, ca, sb, cb);
  __syncthreads();
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int j = R * STB + t;
  if (!half) {
    const float4 hi = shf[t];
    two_sum_acc(sa, ca, hi.x);
    ca += hi.y;
    two_sum_acc(sb, cb, hi.z);
    cb += hi.w;
    if (j < I.n) {
      const size_t o = (size_t)i * I.ldv + j;
      const float u = sa + ca, w = sb + cb;
      U[o] = u;
      W[o] = w;
      const double xj = x[j], vj = v[j], cj = I.c[o];
      dsum[0] = xj * (double)u;
      dsum[1] = vj * (double)w;
      dsum[3] = cj * xj;
      dsum[4] = cj * vj;
    }
  }
  __syncthreads();   // shf is read
  if (!half) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) sh[q * STB + t] = dsum[q];
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  if (warp < NDOT) {
    const double* r = sh + warp * STB;
    double a = r[lane];
#pragma unroll
    for (int k = 1; k < STB / 32; ++k) a += r[lane + 32 * k];
    a = warp_sum(a);
    if (lane == 0) out[(size_t)warp * T] = a;
  }
  __syncthreads();
}

// One CTA's share of the tile products of a packed pass: tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of the (M x ntile) list.  Each 64 KB tile is
// contiguous: one bulk copy (TMA unit) moves it into a shared-memory stage,
// SNST stages in flight, completed on the stage's mbarrier.  The CTA has
// NTS = 512 threads: warp w takes rows 8w .. 8w+7 of the tile, lane l columns
// 4l .. 4l+3 (row partials halved over the lanes, column partials summed over
// the 16 warps in order: at most 8 + 15 float32 roundings per partial).  The
// stage is refilled as soon as all threads have read it, and the next tile's
// right-hand-side slices are loaded while the current tile is reduced.  No counters and no
// global fences: the row-block reduction runs in the next kernel.  Every wait
// is bounded; on a timeout the CTA sets *err, waits (bounded) for its copies
// in flight and returns.
// `dsm` = [SNST mbarriers (128 B) | 2 x NWS x STB floats | SNST x 64 KB stages].
constexpr int NTS = 512;
constexpr int NWS = NTS / 32;
constexpr int SRW8 = STB / NWS;      // tile rows per warp (8)
static_assert(SRW8 == 8, "warp_rows8 reduces 8 rows per warp");
constexpr int SNST = 3;
constexpr uint32_t STILE = (uint32_t)STB * STB * 4;
__host__ __device__ constexpr size_t sym_smem_bytes() {
  return (size_t)128 + (size_t)2 * NWS * STB * 4 + (size_t)SNST * STILE;
}

// Lane l returns the sum over the 32 lanes of a[r] for r = sym_row8(l) (the
// four lanes that share l >> 2 return the same value).
__device__ __forceinline__ int sym_row8(int lane) {
  return 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
}
__device__ __forceinline__ float warp_rows8(float (&a)[SRW8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = hi ? a[k] : a[k + h];
      const float keep = hi ? a[k + h] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float r = a[0] + __shfl_xor_sync(0xffffffffu, a[0], 2);
  return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

// The slices of a right-hand side v a thread needs for tile (TI, TJ):
// v_J[4l .. 4l+3] and, in lanes 0..7, v_I of row 8w + lane (zero past n).
__device__ __forceinline__ void sym_dslices(const float* __restrict__ v, int n, int TI, int TJ, float (&dj)[4],
                                            float& dil) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = TJ * STB + lane * 4;
  if (c0 + 4 <= n) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(v + c0));
    dj[0] = t.x; dj[1] = t.y; dj[2] = t.z; dj[3] = t.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) dj[e] = (c0 + e < n) ? __ldg(v + c0 + e) : 0.f;
  }
  const int r = TI * STB + warp * SRW8 + lane;
  dil = (lane < SRW8 && r < n) ? __ldg(v + r) : 0.f;
}

// NR right-hand sides r0 (and r1): the products of r_k go to slot set k,
// I.sp + k * M * T * T * STB.
template <int NR>
__device__ __forceinline__ void sym_tiles(const Inst& I, const float* __restrict__ r0, const float* __restrict__ r1,
                                          uint8_t* dsm, int* err) {
  const int T = I.tsym, nt = I.ntile;
  const size_t ldp = (size_t)T * STB;
  const int total = I.M * nt;
  const int first = blockIdx.x, G = gridDim.x;
  if (first >= total) return;
  const int K = (total - first + G - 1) / G;          // tiles of this CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const float* rhs[2] = {r0, r1};
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm);
  float* sred = reinterpret_cast<float*>(dsm + 128);
  uint8_t* stg = dsm + 128 + (size_t)2 * NWS * STB * 4;
  if (tid == 0) {
    for (int k = 0; k < SNST; ++k) mbar_init(&full[k], 1);
    fence_proxy_async();
  }
  __syncthreads();
  // the tiles are read once per pass: first out of L2, so that the slot
  // partials stay there for the row-block kernel
  const uint64_t pol = l2_policy_evict_first();
  auto issue = [&](int k) {   // thread 0: tile k of this CTA -> stage k % SNST
    const int st = k % SNST;
    const size_t it = (size_t)first + (size_t)k * G;
    mbar_expect_tx(&full[st], STILE);
    bulk_g2s_evict_first(stg + (size_t)st * STILE, I.Qp + it * STB * STB, STILE, &full[st], pol);
  };
  if (tid == 0)
    for (int k = 0; k < SNST && k < K; ++k) issue(k);
  auto coords = [&](int k, int& s, int& TI, int& TJ) {
    const int it = first + k * G;
    s = it / nt;
    const int ij = __ldg(I.tij + (it - s * nt));
    TI = ij >> 16;
    TJ = ij & 0xffff;
  };
  int s, TI, TJ;
  coords(0, s, TI, TJ);
  float dj[NR][4], dil[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) sym_dslices(rhs[r], I.n, TI, TJ, dj[r], dil[r]);
  for (int k = 0; k < K; ++k) {
    const int st = k % SNST;
    const bool got = mbar_wait_bounded(&full[st], (uint32_t)((k / SNST) & 1), err);
    if (!__syncthreads_and(got)) {
      if (tid == 0)
        for (int k2 = k; k2 < K && k2 < k + SNST; ++k2)
          mbar_wait_bounded(&full[k2 % SNST], (uint32_t)((k2 / SNST) & 1), err);
      __syncthreads();
      return;
    }
#ifdef RAPDB_CHECKED
    if (!__syncthreads_and(TI >= 0 && TI <= TJ && TJ < T)) {
      if (tid == 0) {
        if (err) atomicCAS(err, 0, CHK_SYM_RANGE);
        for (int k2 = k + 1; k2 < K && k2 < k + SNST; ++k2)
          mbar_wait_bounded(&full[k2 % SNST], (uint32_t)((k2 / SNST) & 1), err);
      }
      __syncthreads();
      return;
    }
#endif
    // this thread's share of the tile: rows 8w .. 8w+7, columns 4l .. 4l+3
    float rp[NR][SRW8], cp[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r) cp[r][0] = cp[r][1] = cp[r][2] = cp[r][3] = 0.f;
    {
      const uint8_t* sp = stg + (size_t)st * STILE + ((size_t)warp * SRW8 * STB + lane * 4) * 4;
      uint4 raw[SRW8];
#pragma unroll
      for (int q = 0; q < SRW8; ++q) raw[q] = *reinterpret_cast<const uint4*>(sp + (size_t)q * STB * 4);
#pragma unroll
      for (int q = 0; q < SRW8; ++q) {
        const float b0 = __uint_as_float(raw[q].x), b1 = __uint_as_float(raw[q].y);
        const float b2 = __uint_as_float(raw[q].z), b3 = __uint_as_float(raw[q].w);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          rp[r][q] = fmaf(b3, dj[r][3], fmaf(b2, dj[r][2], fmaf(b1, dj[r][1], b0 * dj[r][0])));
          const float di = __shfl_sync(0xffffffffu, dil[r], q);
          cp[r][0] = fmaf(b0, di, cp[r][0]);
          cp[r][1] = fmaf(b1, di, cp[r][1]);
          cp[r][2] = fmaf(b2, di, cp[r][2]);
          cp[r][3] = fmaf(b3, di, cp[r][3]);
        }
      }
    }
    __syncthreads();   // the stage is consumed (and sred of the previous tile read)
    if (tid == 0 && k + SNST < K) {
      fence_proxy_async();
      issue(k + SNST);
    }
    const int cs = s, cI = TI, cJ = TJ;
    if (k + 1 < K) {   // the next tile's slices, in flight during the reduction
      coords(k + 1, s, TI, TJ);
#pragma unroll
      for (int r = 0; r < NR; ++r) sym_dslices(rhs[r], I.n, TI, TJ, dj[r], dil[r]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float* Ps = I.sp + ((size_t)r * I.M + cs) * T * ldp;
      const float rv = warp_rows8(rp[r]);
      if (!(lane & 3)) Ps[(size_t)cJ * ldp + (size_t)cI * STB + warp * SRW8 + sym_row8(lane)] = rv;
    }
    if (cI != cJ) {
#pragma unroll
      for (int r = 0; r < NR; ++r)
        *reinterpret_cast<float4*>(sred + (r * NWS + warp) * STB + lane * 4) =
            make_float4(cp[r][0], cp[r][1], cp[r][2], cp[r][3]);
      __syncthreads();
      if (tid < NR * STB) {
        const int r = tid / STB, c0 = tid - r * STB;
        const float* sr = sred + r * NWS * STB + c0;
        float c = sr[0];
#pragma unroll
        for (int w = 1; w < NWS; ++w) c += sr[w * STB];
        I.sp[(((size_t)r * I.M + cs) * T + cI) * ldp + (size_t)cJ * STB + c0] = c;
      }
    }
  }
}

// The right-hand sides of a smoothed-gap pass (the row-streaming pass reads
// the same): the power-iteration vector twice, or the extrapolated point and
// the current iterate.
__device__ __forceinline__ void gap_rhs(const Inst& I, int phase, const float*& x, const float*& v) {
  if (phase == PH_GAPP) {
    x = I.gpf;
    v = x;
  } else {
    x = I.gwf;
    v = I.gzf;
  }
}

// The tile products of a packed pass (kind 1: d; kind 2: the gap pass's two
// right-hand sides); outside such a phase every CTA returns at once.  The row
// blocks, dots and control follow in k_sym_finish.  One persistent CTA per
// SM.
template <int DUMMY>
__global__ void __launch_bounds__(NTS, 1) k_sym_tiles(const Inst* __restrict__ insts, const State* __restrict__ states,
                                                     Ctrl* __restrict__ ctrl) {
  extern __shared__ __align__(128) uint8_t dsm[];
  const Inst& I = insts[0];
  const State& S = states[0];
  const int kind = sym_kind(I, S);
  if (kind == 0) return;
#ifdef RAPDB_CHECKED
  if (dyn_smem_bytes() < (unsigned)sym_smem_bytes()) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  if (kind == 1) {
    sym_tiles<1>(I, I.dv, nullptr, dsm, &ctrl->err);
  } else {
    const float *x, *v;
    gap_rhs(I, S.phase, x, v);
    sym_tiles<2>(I, x, v, dsm, &ctrl->err);
  }
}

// Row-streaming tile of a context with packed tiles: 4 rows x 4 chunks per
// warp (tile variant 1), or 8 rows x 2 chunks (variant 8) for FP8 storage,
// whose 16-byte slices of x and v then serve eight rows.
template <int ST>
constexpr int SYM_ROW_VARIANT = (ST == RAPDB_FP8) ? 8 : 1;
template <int ST>
constexpr int SYM_ROW_RPW = (ST == RAPDB_FP8) ? 8 : 4;
template <int ST>
constexpr int SYM_ROW_UNR = (ST == RAPDB_FP8) ? 2 : 4;

// The row-streaming coupling pass of a context with packed tiles (the tile of
// SYM_ROW_VARIANT), each CTA taking the row-block items blockIdx.x,
// blockIdx.x + gridDim.x, ...; in a phase the packed tiles serve every CTA
// returns at once (k_sym_tiles runs it).  A CTA reaches the control step only
// in its last item (the step needs all other items to have arrived), and a
// CTA that owns no item returns whatever state it reads: the state a control
// step leaves is never a packed trial (only the vector kernel sets
// trial_ready) nor a gap phase (only the vector kernel enters those).
template <int ST>
__global__ void __launch_bounds__(NT, 2) k_pass_sym(const Inst* __restrict__ insts, State* __restrict__ states,
                                                    Ctrl* __restrict__ ctrl, const int* __restrict__ pmap,
                                                    const float* __restrict__ XS, const float* __restrict__ VS) {
  extern __shared__ __align__(128) uint8_t dsm[];
  __shared__ double red[NWARP * NDOT];
  __shared__ int s_dec;
  const Inst& I = insts[0];
  if (sym_kind(I, states[0])) return;
  for (int bid = blockIdx.x; bid < I.M * I.nrb; bid += gridDim.x)
    pass_body<ST, SYM_ROW_RPW<ST>, SYM_ROW_UNR<ST>, 0, 0>(insts, states, ctrl, pmap, XS, VS, dsm, red, s_dec, bid);
}

// Second kernel of a packed pass: one CTA per row block (grid M x T) sums
// the block's slots, forms its products (kind 1: the incremental update; kind
// 2: U = Q x, W = Q v) and goes on to the pass's fixed-order dot reduction
// and control step.  Every CTA reads the phase before it arrives, so none can
// see the state the control step leaves; outside a packed pass all return at
// once.
template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_finish(const Inst* __restrict__ insts, State* __restrict__ states,
                                                   Ctrl* __restrict__ ctrl) {
  __shared__ double red[NWARP * NDOT];
  __shared__ __align__(16) double sh[NDOT * STB];   // (read as float2 / float4 by the slot sums)
  __shared__ int s_dec;
  const Inst& I = insts[0];
  State& S = states[0];
  const int kind = sym_kind(I, S);
  if (kind == 0) return;
  const int T = I.tsym;
#ifdef RAPDB_CHECKED
  if (blockIdx.x >= (unsigned)(I.M * T)) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  const int i = s + I.s_off;
  const int phase = S.phase;
  const float* Ps = I.sp + (size_t)s * T * T * STB;
  double* out = I.spart + (size_t)s * NDOT * T + R;
  if (kind == 1) {
    const float* x = I.xf[S.xcur ^ 1];
    sym_rows(I, Ps, R, i, x, I.xl[S.xcur ^ 1], I.dv, I.U[S.ucur], I.Ulo[S.ucur], I.U[S.ucur ^ 1],
             I.Ulo[S.ucur ^ 1], I.W, out, sh);
    pass_finish(I, S, ctrl, s, i, I.spart, T, phase, true, x, I.dv, red, s_dec);
  } else {
    const float *x, *v;
    gap_rhs(I, phase, x, v);
    sym_rows2(I, Ps, Ps + (size_t)I.M * T * T * STB, R, i, x, v, I.U[S.ucur ^ 1], I.W, out, sh);
    pass_finish(I, S, ctrl, s, i, I.spart, T, phase, false, x, v, red, s_dec);
  }
}

// Stand-alone packed pass (no control), in two kernels like the solver's:
// the tile products, then W = Q_i v and U = uold + W per row block with the
// block's dot partials in spart.  Arrays are (m+1, ldv) bases indexed by the
// constraint row; xl, uol, Ulo may be null.
template <int DUMMY>
__global__ void __launch_bounds__(NTS, 1) k_sym_plain(const Inst* __restrict__ insts, const float* __restrict__ v,
                                                     int* err) {
  extern __shared__ __align__(128) uint8_t dsm[];
#ifdef RAPDB_CHECKED
  if (dyn_smem_bytes() < (unsigned)sym_smem_bytes()) {
    if (threadIdx.x == 0 && err) atomicCAS(err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  sym_tiles<1>(insts[0], v, nullptr, dsm, err);
}

template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_rows_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                       const float* __restrict__ xl, const float* __restrict__ v,
                                                       const float* __restrict__ uoh, const float* __restrict__ uol,
                                                       float* __restrict__ U, float* __restrict__ Ulo,
                                                       float* __restrict__ W, double* __restrict__ spart) {
  __shared__ __align__(16) double sh[NDOT * STB];   // (read as float2 / float4 by the slot sums)
  const Inst& I = insts[0];
  const int T = I.tsym;
  if (blockIdx.x >= (unsigned)(I.M * T)) return;
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  sym_rows(I, I.sp + (size_t)s * T * T * STB, R, s + I.s_off, x, xl, v, uoh, uol, U, Ulo, W,
           spart + (size_t)s * NDOT * T + R, sh);
}

}  // namespace rapdb_dev
