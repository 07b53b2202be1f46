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

#include "rapdb_tc.cuh"

namespace rapdb_dev {

constexpr int STB = 128;             // tile edge (rows of a row block)
static_assert(NT == 2 * STB, "the row-block reduction splits the T slots over two halves of the CTA");

// The passes the packed tiles serve: 1 = the incremental compensated trial
// pass (U' = U^k + Q d, one right-hand side) over the float32 tiles, 2 = a
// smoothed-gap pass over the float32 tiles (U = Q x, W = Q v, plain float32
// products, two right-hand sides), 3 = the incremental trial pass of the
// quantised level (U' = U^k + Q~ d over the BF16 / FP8 tiles); 0 = any other
// pass (the row-streaming tile runs it).
__device__ __forceinline__ int sym_kind(const Inst& I, const State& S) {
  if (I.tsym == 0) return 0;
  const int ph = S.phase;
  if (ph == PH_TRIAL) {
    if (!S.trial_ready) return 0;
    if (S.precision == 2) return 1;
    if (S.precision == 3 && I.Qpq) return 3;
    return 0;
  }
  if (gap_phase(ph)) return (I.storage == RAPDB_F32 || S.precision >= 1) ? 2 : 0;
  return 0;
}

// Row block R of stored matrix s (constraint row i) is complete: sum its T
// slots in slot order, apply the incremental update and write the block's dot
// partials to out[q * T].  The slot sums are compensated float32 sums
// (Knuth's TwoSum per addition, the rounding errors summed alongside): within
// 2u of the exact sum plus O(T^2 u^2) of the sum of |slots|.  The two halves
// of the CTA take half the slots each; the low half's sum absorbs the high
// half's with one more TwoSum.  The update u = U^k + w and the five dots run
// in double-float arithmetic on the float32 pipe (float64 runs at a small
// fraction of the float32 rate on this GPU): the per-row products are
// TwoProducts, summed over the block's 128 rows by compensated accumulation
// and a fixed lane / warp tree, and only the block's five sums become
// float64.  xl, uol and Uol may be null (zero low parts, no low output);
// rscale (FP8 tiles) multiplies the slot sums by the matrix's row scales.
// `sh` = NDOT x STB doubles of shared memory (its first 2.2 KB are used).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float a) {
  const float t = s + a;
  const float z = t - s;
  c += (s - (t - z)) + (a - z);
  s = t;
}

// The block's five double-float dot partials (valid in warps 0..3, the low
// half) -> out[q * T] as pairs, in a fixed order.
__device__ __forceinline__ void sym_dots_out(dflt (&dq)[NDOT], float2* __restrict__ out, int T, double* sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* shd = reinterpret_cast<float2*>(sh + 2 * STB);   // NDOT x 4 pairs, after the 2 KB slot exchange area
  if (tid < STB) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) {
      const dflt r = df_warp_sum(dq[q]);
      if (lane == 0) shd[q * 4 + warp] = make_float2(r.hi, r.lo);
    }
  }
  __syncthreads();
  if (tid < NDOT) {
    dflt a = {shd[tid * 4].x, shd[tid * 4].y};
#pragma unroll
    for (int w = 1; w < STB / 32; ++w) a = df_add(a, dflt{shd[tid * 4 + w].x, shd[tid * 4 + w].y});
    out[(size_t)tid * T] = make_float2(a.hi, a.lo);
  }
  __syncthreads();   // sh is reused by the caller
}

static __device__ void sym_rows(const Inst& I, const float* __restrict__ Ps, int R, int i,
                                const float* __restrict__ x, const float* __restrict__ xl,
                                const float* __restrict__ v, const float* __restrict__ uoh,
                                const float* __restrict__ uol, float* __restrict__ Uoh, float* __restrict__ Uol,
                                float* __restrict__ W, float2* __restrict__ out, double* sh,
                                const float* __restrict__ rscale = nullptr) {
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
  dflt dq[NDOT] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int j = R * STB + t;
  if (!half) {
    const float2 hi = shf[t];
    two_sum_acc(sa, ca, hi.x);
    ca += hi.y;
    if (j < I.n) {
      const size_t o = (size_t)i * I.ldv + j;
      dflt w = df_norm(sa, ca);
      if (rscale) {   // FP8 tiles: the slot sums are C (s .* d); w_j = s_j (C (s .* d))_j
        dflt ws = {0.f, 0.f};
        df_acc_mulf(ws, w, rscale[j]);
        w = df_norm(ws.hi, ws.lo);
      }
      const dflt uo = {uoh[o], uol ? uol[o] : 0.f};
      const dflt u = df_add(uo, w);
      Uoh[o] = u.hi;
      if (Uol) Uol[o] = u.lo;
      W[o] = w.hi;
      const dflt xj = {x[j], xl ? xl[j] : 0.f};
      const float vj = v[j], cj = I.c[o];
      df_acc_mul(dq[0], xj, u);
      df_acc_mulf(dq[1], w, vj);
      df_acc_mulf(dq[2], uo, vj);
      df_acc_mulf(dq[3], xj, cj);
      const float p = __fmul_rn(cj, vj);
      df_acc(dq[4], p, __fmaf_rn(cj, vj, -p));
    }
  }
  sym_dots_out(dq, out, T, sh);
}

// The same for a two-right-hand-side pass (kind 2): U = Q_i x and W = Q_i v
// from the two slot sets Px, Pv (compensated float32 slot sums, one final
// rounding each), dots x'U, v'W, 0, c'x, c'v of the float32 values, summed
// as exact TwoProducts in double-float.
static __device__ void sym_rows2(const Inst& I, const float* __restrict__ Px, const float* __restrict__ Pv, int R,
                                 int i, const float* __restrict__ x, const float* __restrict__ v,
                                 float* __restrict__ U, float* __restrict__ W, float2* __restrict__ out, double* sh) {
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
  dflt dq[NDOT] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
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
      const float xj = x[j], vj = v[j], cj = I.c[o];
      float p = __fmul_rn(xj, u);
      df_acc(dq[0], p, __fmaf_rn(xj, u, -p));
      p = __fmul_rn(vj, w);
      df_acc(dq[1], p, __fmaf_rn(vj, w, -p));
      p = __fmul_rn(cj, xj);
      df_acc(dq[3], p, __fmaf_rn(cj, xj, -p));
      p = __fmul_rn(cj, vj);
      df_acc(dq[4], p, __fmaf_rn(cj, vj, -p));
    }
  }
  sym_dots_out(dq, out, T, sh);
}

// One CTA's share of the tile products of a packed pass: tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of the (M x ntile) list.  Each tile (64 KB of
// float32, 32 KB of BF16 or 16 KB of FP8 codes) is contiguous: one bulk copy
// (TMA unit) moves it into a shared-memory stage, 3 / 6 / 12 stages in
// flight, completed on the stage's mbarrier.  The CTA has
// NTS = 512 threads: warp w takes rows 8w .. 8w+7 of the tile, lane l columns
// 4l .. 4l+3 (row partials halved over the lanes, column partials summed over
// the 16 warps in order: at most 8 + 15 float32 roundings per partial).  The
// stage is refilled as soon as all threads have read it, and the next tile's
// right-hand-side slices are loaded while the current tile is reduced.  No counters and no
// global fences: the row-block reduction runs in the next kernel.  Every wait
// is bounded; on a timeout the CTA sets *err, waits (bounded) for its copies
// in flight and returns.
// `dsm` = [stage mbarriers (128 B) | 2 x NWS x STB floats | 192 KB of stages]
// (within sym_smem_bytes(), which the tensor-core path lays out its own way).
constexpr int NTS = 512;
constexpr int NWS = NTS / 32;
constexpr int SRW8 = STB / NWS;      // tile rows per warp (8)
static_assert(SRW8 == 8, "warp_rows8 reduces 8 rows per warp");
constexpr int SNST = 3;                          // float32 stages of 64 KB
constexpr uint32_t STILE = (uint32_t)STB * STB * 4;
// (the tensor-core tile path lays out the same bytes as [barriers 256 B |
// pieces ring 24 KB | stages | zero block 2 KB | metadata 256 B])
__host__ __device__ constexpr size_t sym_smem_bytes() {
  return (size_t)256 + 24576 + (size_t)SNST * STILE + 2048 + 256;
}
static_assert(2 * NWS * STB * 4 <= 24576, "the float32 path's column sums fit before the stages");
// Bytes of one block of right-hand-side pieces (128 entries, eb-byte type).
__host__ __device__ constexpr uint32_t sym_piece_bytes(int eb) { return (uint32_t)(STB * eb / 16) * 128; }

// Stored tile elements.  Float32 tiles are row-major; a thread of the
// CUDA-core tile loop reads 4 consecutive entries of each of its 8 rows (16
// bytes) and decodes them to float32.  The quantised tiles (BF16 / FP8 codes,
// read by the tensor cores) are in the core-matrix layout of rapdb_tc.cuh and
// use the same 192 KB of stages: more, smaller stages in flight.
template <int ST> struct TileElt;
template <> struct TileElt<RAPDB_F32> {
  using raw = uint4;
  static constexpr int B = 4;
  __device__ __forceinline__ static void dec(const raw& r, float (&o)[4]) {
    o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
    o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
  }
};
template <> struct TileElt<RAPDB_BF16> { static constexpr int B = 2; };
template <> struct TileElt<RAPDB_FP8> { static constexpr int B = 1; };
template <int ST>
__host__ __device__ constexpr uint32_t sym_tile_bytes() { return (uint32_t)STB * STB * TileElt<ST>::B; }
template <int ST>
__host__ __device__ constexpr int sym_stages() { return SNST * 4 / TileElt<ST>::B; }
static_assert(sym_stages<RAPDB_FP8>() * 8 <= 128, "mbarriers of the stages fit their 128-byte area");

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
// I.sp + k * M * T * T * STB.  ST selects the tiles: the float32 ones (I.Qp)
// or the quantised ones (I.Qpq, BF16 or FP8 codes).  The right-hand side of
// stored matrix s is r + s * rstride (FP8: its pre-scaled copy s_s .* d;
// otherwise rstride = 0).
// Tile t of the upper block triangle (row-major over I <= J, the order of
// the tile table): row I is the largest with I T - I(I-1)/2 <= t.  Computed
// from t (a float square root, then an exact integer correction), so the
// tile loop issues no dependent table load.
__device__ __forceinline__ void sym_tile_coords(int t, int T, int& TI, int& TJ) {
  const float b = 2.0f * (float)T + 1.0f;
  int i = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)t, 0.0f))));
  i = max(0, min(i, T - 1));
  auto off = [&](int r) { return r * T - (r * (r - 1)) / 2; };
  while (i > 0 && off(i) > t) --i;
  while (i + 1 < T && off(i + 1) <= t) ++i;
  TI = i;
  TJ = i + (t - off(i));
}

template <int NR, int ST>
__device__ __forceinline__ void sym_tiles(const Inst& I, const float* __restrict__ r0, const float* __restrict__ r1,
                                          size_t rstride, uint8_t* dsm, int* err) {
  using TE = TileElt<ST>;
  constexpr uint32_t TB = sym_tile_bytes<ST>();
  constexpr int NSG = sym_stages<ST>();
  // the instance's fields in registers (re-reading them after each barrier
  // would put a dependent load into every tile)
  const uint8_t* Qt = (ST == RAPDB_F32) ? reinterpret_cast<const uint8_t*>(I.Qp)
                                        : reinterpret_cast<const uint8_t*>(I.Qpq);
  const int T = I.tsym, nt = I.ntile, M = I.M, n = I.n;
  float* const sp = I.sp;
  const size_t ldp = (size_t)T * STB;
  const int total = M * nt;
  const int first = blockIdx.x, G = gridDim.x;
  if (first >= total) return;
  const int K = (total - first + G - 1) / G;          // tiles of this CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const float* rhs[2] = {r0, r1};
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm);
  float* sred = reinterpret_cast<float*>(dsm + 128);
  uint8_t* stg = dsm + 128 + (size_t)2 * NWS * STB * 4;
  if (tid == 0) {
    for (int k = 0; k < NSG; ++k) mbar_init(&full[k], 1);
    fence_proxy_async();
  }
  __syncthreads();
  // the tiles are read once per pass: first out of L2, so that the slot
  // partials stay there for the row-block kernel
  const uint64_t pol = l2_policy_evict_first();
  auto issue = [&](int k) {   // thread 0: tile k of this CTA -> stage k % NSG
    const int st = k % NSG;
    const size_t it = (size_t)first + (size_t)k * G;
    mbar_expect_tx(&full[st], TB);
    bulk_g2s_evict_first(stg + (size_t)st * TB, Qt + it * TB, TB, &full[st], pol);
  };
  if (tid == 0)
    for (int k = 0; k < NSG && k < K; ++k) issue(k);
  auto coords = [&](int k, int& s, int& TI, int& TJ) {
    const int it = first + k * G;
    s = it / nt;
    sym_tile_coords(it - s * nt, T, TI, TJ);
  };
  // right-hand-side slices two tiles ahead: those of tile k (cur) and k + 1 (nxt)
  int s, TI, TJ, ns = 0, nI = 0, nJ = 0;
  coords(0, s, TI, TJ);
  float dj[NR][4], dil[NR], nj[NR][4], nil[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) sym_dslices(rhs[r] + (size_t)s * rstride, n, TI, TJ, dj[r], dil[r]);
  if (K > 1) {
    coords(1, ns, nI, nJ);
#pragma unroll
    for (int r = 0; r < NR; ++r) sym_dslices(rhs[r] + (size_t)ns * rstride, n, nI, nJ, nj[r], nil[r]);
  }
  for (int k = 0; k < K; ++k) {
    const int st = k % NSG;
    // (this barrier also ends the previous tile's column sums: sred is free)
    const bool got = mbar_wait_bounded(&full[st], (uint32_t)((k / NSG) & 1), err);
    if (!__syncthreads_and(got)) {
      if (tid == 0)
        for (int k2 = k; k2 < K && k2 < k + NSG; ++k2)
          mbar_wait_bounded(&full[k2 % NSG], (uint32_t)((k2 / NSG) & 1), err);
      __syncthreads();
      return;
    }
#ifdef RAPDB_CHECKED
    if (!__syncthreads_and(TI >= 0 && TI <= TJ && TJ < T)) {
      if (tid == 0) {
        if (err) atomicCAS(err, 0, CHK_SYM_RANGE);
        for (int k2 = k + 1; k2 < K && k2 < k + NSG; ++k2)
          mbar_wait_bounded(&full[k2 % NSG], (uint32_t)((k2 / NSG) & 1), err);
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
      const uint8_t* stp = stg + (size_t)st * TB + ((size_t)warp * SRW8 * STB + lane * 4) * TE::B;
      typename TE::raw raw[SRW8];
#pragma unroll
      for (int q = 0; q < SRW8; ++q)
        raw[q] = *reinterpret_cast<const typename TE::raw*>(stp + (size_t)q * STB * TE::B);
#pragma unroll
      for (int q = 0; q < SRW8; ++q) {
        float bq[4];
        TE::dec(raw[q], bq);
        const float b0 = bq[0], b1 = bq[1], b2 = bq[2], b3 = bq[3];
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
    const bool offd = TI != TJ;
    if (offd) {   // column partials of an off-diagonal tile, summed over the warps below
#pragma unroll
      for (int r = 0; r < NR; ++r)
        *reinterpret_cast<float4*>(sred + (r * NWS + warp) * STB + lane * 4) =
            make_float4(cp[r][0], cp[r][1], cp[r][2], cp[r][3]);
    }
    __syncthreads();   // the stage is consumed and the column partials are in sred
    if (tid == 0 && k + NSG < K) {
      fence_proxy_async();
      issue(k + NSG);
    }
    const int cs = s, cI = TI, cJ = TJ;
    // advance the slices: tile k + 1's are in flight already, tile k + 2's start now
    s = ns;
    TI = nI;
    TJ = nJ;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      dil[r] = nil[r];
#pragma unroll
      for (int e = 0; e < 4; ++e) dj[r][e] = nj[r][e];
    }
    if (k + 2 < K) {
      coords(k + 2, ns, nI, nJ);
#pragma unroll
      for (int r = 0; r < NR; ++r) sym_dslices(rhs[r] + (size_t)ns * rstride, n, nI, nJ, nj[r], nil[r]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float* Ps = sp + ((size_t)r * M + cs) * T * ldp;
      const float rv = warp_rows8(rp[r]);
      if (!(lane & 3)) Ps[(size_t)cJ * ldp + (size_t)cI * STB + warp * SRW8 + sym_row8(lane)] = rv;
    }
    if (offd && tid < NR * STB) {
      const int r = tid / STB, c0 = tid - r * STB;
      const float* sr = sred + r * NWS * STB + c0;
      float v[NWS];
#pragma unroll
      for (int w = 0; w < NWS; ++w) v[w] = sr[w * STB];
      float c = v[0];
#pragma unroll
      for (int w = 1; w < NWS; ++w) c += v[w];
      sp[(((size_t)r * M + cs) * T + cI) * ldp + (size_t)cJ * STB + c0] = c;
    }
  }
}

// The quantised tiles (BF16 / FP8 codes, one right-hand side) on the
// tensor cores.  On the CUDA cores a quantised tile costs as much
// arithmetic as a float32 one (decode, then two FMAs per entry, plus the
// shuffle and shared-memory reductions) in a half or a quarter of the bytes:
// measured, that kernel was issue-bound at about 4 TB/s of BF16 and 2 TB/s of
// FP8 tiles.  Here each tile is two small MMAs of the fifth-generation tensor
// cores, operands in shared memory, accumulators in tensor memory (TMEM):
//   row product    D_r (128 x 16) = B  P_J   (B = the tile, read K-major),
//   column product D_c (128 x 16) = B' P_I   (the same tile, read MN-major),
// the quantised tiles being stored in the core-matrix layout (8 rows x 16
// bytes per 128-byte core, cores row-major over the tile), which both
// readings accept.  P_J holds the right-hand side's slice d_J split into
// pieces of the tile's own type, one piece per column of the N = 16 operand,
// so that the products of the pieces are exact and only the float32
// accumulation rounds:
//   BF16: d = h + m + l, three bf16 pieces (exact: 3 x 8 significant bits,
//         for |d| >= 2^-100);
//   FP8:  sigma d = sum_j q_j 16^-j, six e4m3 pieces, sigma a power of two per
//         128-entry slice (|sigma d| < 256), each residual scaled by 16 before
//         it is rounded; the pieces hold sigma d to 2^-23 of each entry or
//         2^-37 of the slice's largest entry, whichever is larger.
// The pieces are formed once per pass (sym_pieces, in the kernel that runs
// before the tile kernel) into blocks of one 128-entry slice each; each
// tile's stage receives its tile and the blocks of slices J and I by bulk
// copy on one mbarrier.  Operand rows 8-15 are an all-zero block in shared
// memory (the descriptors' SBO points there).  The epilogue adds the pieces'
// columns (Horner in 1/16, then 1/sigma, for FP8) and writes the tile's row
// and column partials to their slots, as the float32 tile kernel does.
//
// Warp roles (NTS = 512 threads), linked by mbarriers, no CTA barrier per
// tile:
//   producer (warp 9; its elected lane issues): waits until the MMAs of the
//     stage's previous tile are done (empty), then copies tile k and its
//     pieces blocks (full);
//   MMA issuer (warp 8; its elected lane issues): waits for the stage (full)
//     and for the accumulator pair of tile k - TC_NACC to be read out
//     (accempty), issues the row and column MMAs, then commits them to
//     accfull;
//   epilogue (warps 0-7): waits for accfull, takes FP8's 1 / sigma from the
//     stage's pieces and frees the stage (empty, one arrival per warp), reads
//     its accumulators (warps 0-3 the row products, TMEM lanes 32 w ..;
//     warps 4-7 the column products), arrives on accempty, adds the pieces'
//     columns and stores.
// Each role derives the tile coordinates it needs from k (the issuer reads
// the producer's, published by the full barrier's arrival).
// TMEM: 128 columns, four tiles of [row 16 | column 16] in flight between
// the issuer and the epilogue.  Every wait is bounded and also gives up when
// another role has failed; on a failure the CTA sets *err, drains its copies
// and MMAs in flight (bounded), frees its TMEM and returns.
constexpr int TC_MMA = 8 * 32;              // warp 8 (lane 0 issues)
constexpr int TC_PROD = 9 * 32;             // warp 9
constexpr int TC_NACC = 4;                  // accumulator pairs
constexpr int TC_NCOL = 32 * TC_NACC;
struct TcMeta {
  uint32_t tmem;
  int fail;                    // a role's wait gave up
  int issued;                  // tiles whose copies the producer issued
  int ti[16], tj[16];          // tile k's coordinates in slot k % 16 (written before its copies)
};
// tensor-core layout: [barriers 256 B | pieces ring | stages | zero block | metadata]
constexpr size_t TC_BARS = 256;
constexpr size_t TC_PRING = 24576;
constexpr size_t TC_ZERO = 2048;
static_assert(sizeof(TcMeta) <= 256, "tile metadata fits the tail of the shared-memory layout");
static_assert(TC_BARS + TC_PRING + (size_t)SNST * STILE + TC_ZERO + 256 == sym_smem_bytes(), "shared layout");

// A bounded wait that also gives up once *fail is set.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, int* err, const int* fail) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*reinterpret_cast<const volatile int*>(fail)) return false;
      if (globaltimer() - t0 > 2000000000ull) {
        if (err) atomicExch(err, 1);
        return false;
      }
    }
  }
}

// Pieces of one 128-entry slice e (lane l holds entries 4l .. 4l+3) into the
// block P: core kc (128 bytes) holds entries kc CE .. kc CE + CE - 1, row j
// of the core their piece j.  FP8 also stores 1 / sigma in row 7 of core 0
// (operand row 7 meets D column 7, which nothing reads).
template <int ST>
__device__ __forceinline__ void sym_piece_block(float4 e, uint8_t* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  float a0 = e.x, a1 = e.y, a2 = e.z, a3 = e.w;
  if constexpr (ST == RAPDB_BF16) {
    uint8_t* p = P + (lane >> 1) * 128 + (lane & 1) * 8;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(a0, a1);
      const __nv_bfloat162 hi = __floats2bfloat162_rn(a2, a3);
      *reinterpret_cast<uint2*>(p + j * 16) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
      // exact: the residual of a rounding to 8 significant bits
      a0 -= __low2float(lo);
      a1 -= __high2float(lo);
      a2 -= __low2float(hi);
      a3 -= __high2float(hi);
    }
  } else {
    float mx = fmaxf(fmaxf(fabsf(a0), fabsf(a1)), fmaxf(fabsf(a2), fabsf(a3)));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int ex = 0;
    (void)frexpf(mx, &ex);                                    // mx < 2^ex
    ex = max(-100, min(ex, 100));
    const float sig = __int_as_float((127 + 8 - ex) << 23);  // 2^(8 - ex): |sigma e| < 256
    a0 *= sig;
    a1 *= sig;
    a2 *= sig;
    a3 *= sig;
    uint8_t* p = P + (lane >> 2) * 128 + (lane & 3) * 4;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a0, a1), __NV_SATFINITE, __NV_E4M3);
      const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(a2, a3), __NV_SATFINITE, __NV_E4M3);
      *reinterpret_cast<uint32_t*>(p + j * 16) = (uint32_t)lo | ((uint32_t)hi << 16);
      __half2_raw hl = __nv_cvt_fp8x2_to_halfraw2(lo, __NV_E4M3);
      __half2_raw hh = __nv_cvt_fp8x2_to_halfraw2(hi, __NV_E4M3);
      const float2 ql = __half22float2(*reinterpret_cast<__half2*>(&hl));
      const float2 qh = __half22float2(*reinterpret_cast<__half2*>(&hh));
      // exact: the e4m3 value is a multiple of the residual's float32 ulp
      a0 = (a0 - ql.x) * 16.0f;
      a1 = (a1 - ql.y) * 16.0f;
      a2 = (a2 - qh.x) * 16.0f;
      a3 = (a3 - qh.y) * 16.0f;
    }
    if (lane == 0) *reinterpret_cast<float*>(P + 7 * 16) = __int_as_float((127 - 8 + ex) << 23);   // 1 / sigma
  }
}

// All piece blocks of a pass's right-hand side, one warp per block: BF16 the
// T slices of r, FP8 the M x T slices of r + s rstride (s_s .* d).
template <int ST>
__device__ __forceinline__ void sym_pieces(const Inst& I, const float* __restrict__ r, size_t rstride) {
  constexpr uint32_t PB = sym_piece_bytes(TileElt<ST>::B);
  const int T = I.tsym, n = I.n;
  const int nb = (ST == RAPDB_FP8 ? I.M : 1) * T;
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int q = blockIdx.x * nw + (threadIdx.x >> 5); q < nb; q += gridDim.x * nw) {
    const int s = q / T, b = q - s * T;
    const float* v = r + (size_t)s * rstride;
    const int c0 = b * STB + lane * 4;
    float4 e;
    if (c0 + 4 <= n) {
      e = __ldg(reinterpret_cast<const float4*>(v + c0));
    } else {
      e.x = (c0 < n) ? __ldg(v + c0) : 0.f;
      e.y = (c0 + 1 < n) ? __ldg(v + c0 + 1) : 0.f;
      e.z = (c0 + 2 < n) ? __ldg(v + c0 + 2) : 0.f;
      e.w = (c0 + 3 < n) ? __ldg(v + c0 + 3) : 0.f;
    }
    sym_piece_block<ST>(e, I.Pq + (size_t)q * PB);
  }
}

template <int ST>
__device__ __forceinline__ void sym_tiles_tc(const Inst& I, uint8_t* dsm, int* err) {
  constexpr bool F8 = (ST == RAPDB_FP8);
  constexpr uint32_t TB = sym_tile_bytes<ST>();
  constexpr uint32_t PB = sym_piece_bytes(TileElt<ST>::B);
  constexpr int NSG = sym_stages<ST>();
  static_assert(NSG * 2 * PB <= TC_PRING && NSG <= 12 && PB <= TC_ZERO, "tensor-core stage layout");
  constexpr uint32_t NC = STB * TileElt<ST>::B / 16;     // cores per core row of a tile
  constexpr int KSTEPS = F8 ? 4 : 8;                     // MMAs per product (K = 32 / 16 each)
  constexpr uint32_t IDR = umma_idesc(F8, false, STB, 16), IDC = umma_idesc(F8, true, STB, 16);
  const uint8_t* Qt = reinterpret_cast<const uint8_t*>(I.Qpq);
  const uint8_t* Pq = I.Pq;
  const int T = I.tsym, nt = I.ntile;
  float* const sp = I.sp;
  const size_t ldp = (size_t)T * STB;
  const int total = I.M * nt;
  const int first = blockIdx.x, G = gridDim.x;
  if (first >= total) return;
  const int K = (total - first + G - 1) / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
#ifdef RAPDB_CHECKED
  {
    bool bad = false;
    for (int k = 0; k < K && !bad; ++k) {
      const int it = first + k * G, s = it / nt;
      int TI, TJ;
      sym_tile_coords(it - s * nt, T, TI, TJ);
      bad = TI < 0 || TI > TJ || TJ >= T || s >= I.M;
    }
    if (bad) {
      if (tid == 0 && err) atomicCAS(err, 0, CHK_SYM_RANGE);
      return;
    }
  }
#endif
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm);     // [12]
  uint64_t* empty = full + 12;                           // [12]
  uint64_t* accfull = full + 24;                         // [TC_NACC]
  uint64_t* accempty = full + 24 + TC_NACC;              // [TC_NACC]
  static_assert((24 + 2 * TC_NACC) * 8 <= TC_BARS, "barriers fit their area");
  uint8_t* pring = dsm + TC_BARS;                        // stage st: [P_J | P_I]
  uint8_t* stg = pring + TC_PRING;
  uint8_t* zero = stg + (size_t)SNST * STILE;
  TcMeta* meta = reinterpret_cast<TcMeta*>(zero + TC_ZERO);
  if (tid == 0) {
    for (int k = 0; k < NSG; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 8);           // one arrival per epilogue warp
    }
    for (int b = 0; b < TC_NACC; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 8);        // one arrival per epilogue warp
    }
    fence_proxy_async();
    meta->fail = 0;
    meta->issued = 0;
  }
  for (int i = tid; i < (int)(TC_ZERO / 16); i += NTS) reinterpret_cast<uint4*>(zero)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(&meta->tmem, TC_NCOL);
  fence_proxy_async();   // the zero block is read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = meta->tmem;
  int* const fail = &meta->fail;
  int consumed = 0, committed = -1;                      // (the MMA issuer's)
  if (warp == TC_PROD / 32) {
    const uint64_t pol = l2_policy_evict_first();
    int k = 0;
    for (; k < K; ++k) {
      const int st = k % NSG;
      const int it = first + k * G;
      const int s = it / nt;
      int TI, TJ;
      sym_tile_coords(it - s * nt, T, TI, TJ);
      if (k >= NSG &&
          !__all_sync(0xffffffffu, tc_wait(&empty[st], (uint32_t)(((k / NSG) - 1) & 1), err, fail))) {
        if (lane == 0) *fail = 1;
        break;
      }
      const uint8_t* pb = Pq + (size_t)(F8 ? s : 0) * T * PB;
      const bool off = TI != TJ;
      if (elect_one()) {
        meta->ti[k & 15] = TI;
        meta->tj[k & 15] = TJ;
        mbar_expect_tx(&full[st], TB + PB * (off ? 2u : 1u));
        bulk_g2s_evict_first(stg + (size_t)st * TB, Qt + (size_t)it * TB, TB, &full[st], pol);
        bulk_g2s(pring + (size_t)st * 2 * PB, pb + (size_t)TJ * PB, PB, &full[st]);
        if (off) bulk_g2s(pring + (size_t)st * 2 * PB + PB, pb + (size_t)TI * PB, PB, &full[st]);
      }
      __syncwarp();
    }
    if (lane == 0) meta->issued = k;
  } else if (warp == TC_MMA / 32) {
    const uint32_t zr = smem_u32(zero);
    for (int k = 0; k < K; ++k) {
      const int st = k % NSG, b = k % TC_NACC;
      if (!__all_sync(0xffffffffu, tc_wait(&full[st], (uint32_t)((k / NSG) & 1), err, fail))) {
        if (lane == 0) *fail = 1;
        break;
      }
      consumed = k + 1;
      if (k >= TC_NACC &&
          !__all_sync(0xffffffffu, tc_wait(&accempty[b], (uint32_t)(((k / TC_NACC) - 1) & 1), err, fail))) {
        if (lane == 0) *fail = 1;
        break;
      }
      tc_fence_after();
      // (the producer wrote tile k's coordinates before its copies completed)
      const bool off = meta->ti[k & 15] != meta->tj[k & 15];
      const uint32_t a = smem_u32(stg + (size_t)st * TB);
      const uint32_t pj = smem_u32(pring + (size_t)st * 2 * PB), pi = pj + PB;
      const uint64_t ar = umma_sdesc(a, 128u, NC * 128u), bj = umma_sdesc(pj, 128u, zr - pj);
      const uint64_t ac = umma_sdesc(a, NC * 128u, 128u), bi = umma_sdesc(pi, 128u, zr - pi);
      const uint32_t d = tmem + (uint32_t)b * 32;
      // K steps: the tile's next two cores along the row (256 B) for the row
      // product, its next 16 / 32 rows (4096 B) for the column product; the
      // pieces' next two cores (256 B); addresses in 16-byte units
#pragma unroll
      for (int kk = 0; kk < KSTEPS; ++kk) {
        if (elect_one()) umma<F8>(d, ar + 16u * kk, bj + 16u * kk, IDR, kk > 0);
        __syncwarp();
      }
      if (off) {
#pragma unroll
        for (int kk = 0; kk < KSTEPS; ++kk) {
          if (elect_one()) umma<F8>(d + 16, ac + 256u * kk, bi + 16u * kk, IDC, kk > 0);
          __syncwarp();
        }
      }
      // (the elected lane is the lowest active one: the lane that issued)
      if (elect_one()) umma_commit(&accfull[b]);
      __syncwarp();
      committed = k;
    }
  } else if (warp < 8) {
    const bool rowp = warp < 4;
    const int t = 32 * (warp & 3) + lane;
    // tile coordinates two tiles ahead (off the accumulator read-out)
    struct Ahead {
      int s, ti, tj;
    };
    auto look = [&](int k) {
      Ahead a{0, 0, 0};
      if (k < K) {
        const int it = first + k * G;
        a.s = it / nt;
        sym_tile_coords(it - a.s * nt, T, a.ti, a.tj);
      }
      return a;
    };
    Ahead a0 = look(0), a1 = look(1);
    for (int k = 0; k < K; ++k) {
      const int b = k % TC_NACC;
      const Ahead cur = a0;
      a0 = a1;
      a1 = look(k + 2);
      const int s = cur.s, TI = cur.ti, TJ = cur.tj;
      const bool work = rowp || TI != TJ;
      const bool ok =
          __all_sync(0xffffffffu, tc_wait(&accfull[b], (uint32_t)((k / TC_NACC) & 1), err, fail));
      if (!ok) {
        if (lane == 0) *fail = 1;
        break;
      }
      // tile k's MMAs are done; FP8's 1 / sigma comes from the stage's pieces
      // (its copies completed before the MMAs ran: the full wait returns at
      // once), then this warp releases the stage to the producer
      float sc = 1.0f;
      if constexpr (F8) {
        const int st = k % NSG;
        if (work && __all_sync(0xffffffffu, tc_wait(&full[st], (uint32_t)((k / NSG) & 1), err, fail)))
          sc = *reinterpret_cast<const float*>(pring + (size_t)st * 2 * PB + (rowp ? 0 : PB) + 7 * 16);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[k % NSG]);
      tc_fence_after();
      float v[8];
      if (work) tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)b * 32 + (rowp ? 0u : 16u), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[b]);
      if (work) {
        float y;
        if constexpr (F8) {
          float acc = v[5];
#pragma unroll
          for (int q = 4; q >= 0; --q) acc = fmaf(acc, 0.0625f, v[q]);
          y = acc * sc;
        } else {
          (void)sc;
          y = (v[2] + v[1]) + v[0];
        }
        if (rowp)
          sp[((size_t)s * T + TJ) * ldp + (size_t)TI * STB + t] = y;
        else
          sp[((size_t)s * T + TI) * ldp + (size_t)TJ * STB + t] = y;
      }
    }
  }
  // on a failure, drain this CTA's copies and MMAs in flight
  __syncthreads();
  if (tid == TC_MMA && *reinterpret_cast<volatile int*>(fail)) {
    const int issued = meta->issued;
    for (int k2 = consumed; k2 < issued; ++k2)
      mbar_wait_bounded(&full[k2 % NSG], (uint32_t)((k2 / NSG) & 1), err);
    if (committed >= 0)
      mbar_wait_bounded(&accfull[committed % TC_NACC], (uint32_t)((committed / TC_NACC) & 1), err);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TC_NCOL);
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
// ST is the context's storage: a quantised context's trials at the quantised
// level (kind 3) read its BF16 / FP8 tiles; the FP8 right-hand sides are the
// pre-scaled copies VS (s_s .* d per stored matrix) the vector kernel wrote.
template <int ST>
__global__ void __launch_bounds__(NTS, 1) k_sym_tiles(const Inst* __restrict__ insts, const State* __restrict__ states,
                                                     Ctrl* __restrict__ ctrl, const float* __restrict__ VS) {
  extern __shared__ __align__(128) uint8_t dsm[];
  const Inst& I = insts[0];
  const State& S = states[0];
  const int kind = sym_kind(I, S);
  if (kind == 0) return;
#ifdef RAPDB_CHECKED
  if (dyn_smem_bytes() < (unsigned)sym_smem_bytes() || (kind == 3 && (ST == RAPDB_F32 || I.storage != ST))) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  if (kind == 1) {
    sym_tiles<1, RAPDB_F32>(I, I.dv, nullptr, 0, dsm, &ctrl->err);
  } else if (kind == 2) {
    const float *x, *v;
    gap_rhs(I, S.phase, x, v);
    sym_tiles<2, RAPDB_F32>(I, x, v, 0, dsm, &ctrl->err);
  } else if constexpr (ST != RAPDB_F32) {
    sym_tiles_tc<ST>(I, dsm, &ctrl->err);   // the pieces of d were formed by k_pass_sym
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
  const int kind = sym_kind(I, states[0]);
  if (kind == 3) {   // a trial of the quantised level: the pieces of d for the tile kernel
    if constexpr (ST != RAPDB_F32) sym_pieces<ST>(I, ST == RAPDB_FP8 ? VS : I.dv, ST == RAPDB_FP8 ? (size_t)I.ldv : 0);
    return;
  }
  if (kind) return;
  for (int bid = blockIdx.x; bid < I.M * I.nrb; bid += gridDim.x)
    pass_body<ST, SYM_ROW_RPW<ST>, SYM_ROW_UNR<ST>, 0, 0>(insts, states, ctrl, pmap, XS, VS, dsm, red, s_dec, bid);
}

// Second kernel of a packed pass: one CTA per row block (grid M x T) sums
// the block's slots and forms its products (kind 1 / 3: the incremental
// update; kind 2: U = Q x, W = Q v) and the block's dot partials.  No
// arrival counters and no fences: the third kernel (k_sym_ctrl) reduces the
// partials and runs the control step after the kernel boundary.  Outside a
// packed pass every CTA returns at once.
template <int ST>
__global__ void __launch_bounds__(NT) k_sym_finish(const Inst* __restrict__ insts, State* __restrict__ states,
                                                   Ctrl* __restrict__ ctrl) {
  __shared__ __align__(16) double sh[NDOT * STB];   // (read as float2 / float4 by the slot sums)
  const Inst& I = insts[0];
  const State& S = states[0];
  const int kind = sym_kind(I, S);
  if (kind == 0) return;
  const int T = I.tsym;
#ifdef RAPDB_CHECKED
  if (blockIdx.x >= (unsigned)(I.M * T)) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, CHK_SYM_RANGE);
    return;
  }
#else
  (void)ctrl;
#endif
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  const int i = s + I.s_off;
  const float* Ps = I.sp + (size_t)s * T * T * STB;
  float2* out = I.spart + (size_t)s * NDOT * T + R;
  if (kind == 1 || kind == 3) {
    // kind 3 with FP8 tiles: the slot sums carry the row scales of matrix s
    const float* rs = (kind == 3 && ST == RAPDB_FP8) ? I.qscale + (size_t)s * I.ldv : nullptr;
    sym_rows(I, Ps, R, i, I.xf[S.xcur ^ 1], I.xl[S.xcur ^ 1], I.dv, I.U[S.ucur], I.Ulo[S.ucur], I.U[S.ucur ^ 1],
             I.Ulo[S.ucur ^ 1], I.W, out, sh, rs);
  } else {
    const float *x, *v;
    gap_rhs(I, S.phase, x, v);
    sym_rows2(I, Ps, Ps + (size_t)I.M * T * T * STB, R, i, x, v, I.U[S.ucur ^ 1], I.W, out, sh);
  }
}

// Third kernel of a packed pass (one CTA): each matrix's row-block partials
// summed in row-block order (double-float, one thread per matrix and dot)
// into I.dots, then the pass's control step.
// The control step works on a shared-memory copy of the state (written back
// at the end): its serial scalar updates then cost no global round trips.
constexpr int SYM_CTRL_ROWS = 256;
template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_ctrl(const Inst* __restrict__ insts, State* __restrict__ states,
                                                 Ctrl* __restrict__ ctrl) {
  __shared__ double red[NWARP * NDOT];
  __shared__ int s_dec;
  __shared__ __align__(16) State S;
  __shared__ __align__(16) Inst sI;
  __shared__ double sdots[SYM_CTRL_ROWS * NDOT];
  {
    // the state and the instance descriptor in shared memory: one parallel
    // copy instead of a global round trip per field in the serial steps
    static_assert(sizeof(State) % 4 == 0 && sizeof(Inst) % 4 == 0, "copies in words");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&states[0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&S);
    for (int w = threadIdx.x; w < (int)(sizeof(State) / 4); w += NT) dst[w] = src[w];
    const uint32_t* isrc = reinterpret_cast<const uint32_t*>(&insts[0]);
    uint32_t* idst = reinterpret_cast<uint32_t*>(&sI);
    for (int w = threadIdx.x; w < (int)(sizeof(Inst) / 4); w += NT) idst[w] = isrc[w];
  }
  __syncthreads();
  const Inst& I = sI;
  const int kind = sym_kind(I, S);
  if (kind == 0) return;
  const int T = I.tsym, phase = S.phase;
  // the dots also stay in shared memory for the control step (up to
  // SYM_CTRL_ROWS constraint rows), which then reads them without a round trip
  double* Dsh = (I.m + 1 <= SYM_CTRL_ROWS) ? sdots : nullptr;
  for (int pq = threadIdx.x; pq < I.M * NDOT; pq += NT) {
    const int s = pq / NDOT, q = pq - s * NDOT;
    const double d = df_to_double(df_sum_pairs(I.spart + ((size_t)s * NDOT + q) * T, T));
    I.dots[(size_t)(s + I.s_off) * NDOT + q] = d;
    if (Dsh) Dsh[(s + I.s_off) * NDOT + q] = d;
  }
  __syncthreads();
  if (kind == 2) {
    const float *x, *v;
    gap_rhs(I, phase, x, v);
    pass_control(I, S, ctrl, phase, false, x, v, red, s_dec, Dsh);
  } else {
    pass_control(I, S, ctrl, phase, true, I.xf[S.xcur ^ 1], I.dv, red, s_dec, Dsh);
  }
  __syncthreads();
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&S);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&states[0]);
    for (int w = threadIdx.x; w < (int)(sizeof(State) / 4); w += NT) dst[w] = src[w];
  }
}

// Stand-alone packed pass (no control), in two kernels like the solver's:
// the tile products, then W = Q_i v and U = uold + W per row block with the
// block's dot partials in spart.  Arrays are (m+1, ldv) bases indexed by the
// constraint row; xl, uol, Ulo may be null.  quant = 1 reads the quantised
// tiles of a BF16 / FP8 context (FP8: v is the pre-scaled (M, ldv) array
// s_s .* v and the row-block kernel gets the row scales).
template <int ST>
__global__ void __launch_bounds__(NTS, 1) k_sym_plain(const Inst* __restrict__ insts, const float* __restrict__ v,
                                                     int quant, int* err) {
  extern __shared__ __align__(128) uint8_t dsm[];
#ifdef RAPDB_CHECKED
  if (dyn_smem_bytes() < (unsigned)sym_smem_bytes() || (quant && (ST == RAPDB_F32 || insts[0].storage != ST))) {
    if (threadIdx.x == 0 && err) atomicCAS(err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  if constexpr (ST != RAPDB_F32) {
    if (quant) {
      sym_tiles_tc<ST>(insts[0], dsm, err);   // the pieces of v: k_sym_pieces
      return;
    }
  }
  sym_tiles<1, RAPDB_F32>(insts[0], v, nullptr, 0, dsm, err);
}

// The pieces of a stand-alone pass's right-hand side v for the quantised
// tiles (FP8: v is the pre-scaled (M, ldv) array s_s .* v).
template <int ST>
__global__ void __launch_bounds__(NT) k_sym_pieces(const Inst* __restrict__ insts, const float* __restrict__ v) {
  if constexpr (ST != RAPDB_F32)
    sym_pieces<ST>(insts[0], v, ST == RAPDB_FP8 ? (size_t)insts[0].ldv : 0);
}

template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_rows_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                       const float* __restrict__ xl, const float* __restrict__ v,
                                                       const float* __restrict__ uoh, const float* __restrict__ uol,
                                                       float* __restrict__ U, float* __restrict__ Ulo,
                                                       float* __restrict__ W, float2* __restrict__ spart,
                                                       const float* __restrict__ rscale) {
  __shared__ __align__(16) double sh[NDOT * STB];   // (read as float2 / float4 by the slot sums)
  const Inst& I = insts[0];
  const int T = I.tsym;
  if (blockIdx.x >= (unsigned)(I.M * T)) return;
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  sym_rows(I, I.sp + (size_t)s * T * T * STB, R, s + I.s_off, x, xl, v, uoh, uol, U, Ulo, W,
           spart + (size_t)s * NDOT * T + R, sh, rscale ? rscale + (size_t)s * I.ldv : nullptr);
}

}  // namespace rapdb_dev
