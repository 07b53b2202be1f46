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
// in slot order, in float64, then applies the incremental compensated update
// of the trial pass:
//   w = (Q_i d)_j,  u = U^k_j (double-float) + w,  U' = hi/lo of u,  W = w,
// with the per-row dots x'u, v'w, v'U^k, c'x, c'v.  The tile kernel streams
// with no counters or fences (the kernel boundary orders its stores before
// the reduction), and every sum has a fixed order: runs are bit-for-bit
// reproducible.
//
// The packed pass serves the incremental trials (U' = U^k + Q d at the
// compensated level, the dominant pass of a solve); the direct compensated
// anchors, the setup and check passes and the smoothed gap's passes keep the
// row-streaming tile.
#pragma once

namespace rapdb_dev {

constexpr int STB = 128;             // tile edge (rows of a row block)
constexpr int SRW = STB / NWARP;     // tile rows per warp
static_assert(NT == 2 * STB, "the row-block reduction splits the T slots over two halves of the CTA");
static_assert(SRW == 16, "warp_rows16 reduces 16 rows per warp");
static_assert(STB == 32 * 4, "one float4 column slice per lane");

// The incremental compensated trial pass (the phase the packed tiles serve).
__device__ __forceinline__ bool sym_phase(const Inst& I, const State& S) {
  return I.tsym > 0 && S.phase == PH_TRIAL && S.trial_ready && S.precision == 2 && S.anchor_age < ANCHOR_EVERY;
}

// Issue the SRW 16-byte loads of this thread's share of a tile: warp w reads
// rows w*SRW .. w*SRW+SRW-1, lane l columns 4l .. 4l+3 (each row one 512-byte
// coalesced load per warp).
__device__ __forceinline__ void sym_load(const float* tile, uint4 (&raw)[SRW]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint8_t* p = reinterpret_cast<const uint8_t*>(tile + (size_t)warp * SRW * STB + lane * 4);
#pragma unroll
  for (int q = 0; q < SRW; ++q) raw[q] = ld_stream16(p + (size_t)q * STB * 4);
}

// Row partials rp[q] = B[q, 4l..4l+3] . d_J[4l..4l+3] and column partials
// cp[e] = sum_q d_I[q] B[q, 4l+e] of this thread's share of tile (I, J).
__device__ __forceinline__ void sym_compute(const uint4 (&raw)[SRW], int TI, int TJ, int n,
                                            const float* __restrict__ v, float (&rp)[SRW], float (&cp)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = TJ * STB + lane * 4;
  float dj[4];
  if (c0 + 4 <= n) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(v + c0));
    dj[0] = t.x; dj[1] = t.y; dj[2] = t.z; dj[3] = t.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) dj[e] = (c0 + e < n) ? __ldg(v + c0 + e) : 0.f;
  }
  const int r0 = TI * STB + warp * SRW;
  const float dil = (lane < SRW && r0 + lane < n) ? __ldg(v + r0 + lane) : 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) cp[e] = 0.f;
#pragma unroll
  for (int q = 0; q < SRW; ++q) {
    const float b0 = __uint_as_float(raw[q].x), b1 = __uint_as_float(raw[q].y);
    const float b2 = __uint_as_float(raw[q].z), b3 = __uint_as_float(raw[q].w);
    rp[q] = fmaf(b3, dj[3], fmaf(b2, dj[2], fmaf(b1, dj[1], b0 * dj[0])));
    const float di = __shfl_sync(0xffffffffu, dil, q);
    cp[0] = fmaf(b0, di, cp[0]);
    cp[1] = fmaf(b1, di, cp[1]);
    cp[2] = fmaf(b2, di, cp[2]);
    cp[3] = fmaf(b3, di, cp[3]);
  }
}

// Sum of a[0..15] over the warp's 32 lanes by halving: at each step a lane
// keeps half of its rows and adds its partner's copy of them.  Lane l returns
// the sum for row sym_row(l); lanes l and l ^ 1 return the same value.
__device__ __forceinline__ int sym_row(int lane) {
  return 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
}
__device__ __forceinline__ float warp_rows16(float (&a)[SRW]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = hi ? a[k] : a[k + h];
      const float keep = hi ? a[k + h] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// Row block R of stored matrix s (constraint row i) is complete: sum its T
// slots in slot order (float64; the two halves of the CTA take half the slots
// each, added low half first), apply the incremental update and write the
// block's dot partials to out[q * T].  xl, uol and Uol may be null (zero low
// parts, no low output).
static __device__ void sym_rows(const Inst& I, const float* __restrict__ Ps, int R, int i,
                                const float* __restrict__ x, const float* __restrict__ xl,
                                const float* __restrict__ v, const float* __restrict__ uoh,
                                const float* __restrict__ uol, float* __restrict__ Uoh, float* __restrict__ Uol,
                                float* __restrict__ W, double* __restrict__ out, double* sh, double* red) {
  const int T = I.tsym;
  const size_t ldp = (size_t)T * STB;
  const int tid = threadIdx.x, t = tid & (STB - 1), half = tid / STB;
  const int h = T / 2;
  const int s0 = half ? h : 0, s1 = half ? T : h;
  const float* src = Ps + (size_t)R * STB + t;
  double w = 0.0;
#pragma unroll 4
  for (int sl = s0; sl < s1; ++sl) w += (double)__ldcg(src + (size_t)sl * ldp);
  if (half) sh[t] = w;
  __syncthreads();
  double dsum[NDOT] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int j = R * STB + t;
  if (!half && j < I.n) {
    w += sh[t];
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
  block_sum<NDOT>(dsum, red);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q) out[(size_t)q * T] = dsum[q];
  }
}

// One CTA's share of the tile products of a packed pass: tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of the (M x ntile) list, the loads of the next
// tile in flight while the current one is reduced and stored.  No counters
// and no fences: the row-block reduction runs in the next kernel.
__device__ __forceinline__ void sym_tiles(const Inst& I, const float* __restrict__ v, float* sred, int* err) {
  const int T = I.tsym, nt = I.ntile;
  const size_t ldp = (size_t)T * STB;
  const int total = I.M * nt;
  int it = blockIdx.x;
  if (it >= total) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  uint4 raw[SRW];
  sym_load(I.Qp + (size_t)it * STB * STB, raw);
  for (;;) {
    const int s = it / nt, t = it - s * nt;
    const int ij = __ldg(I.tij + t);
    const int TI = ij >> 16, TJ = ij & 0xffff;
#ifdef RAPDB_CHECKED
    if (!(TI >= 0 && TI <= TJ && TJ < T)) {
      if (tid == 0 && err) atomicCAS(err, 0, CHK_SYM_RANGE);
      return;
    }
#else
    (void)err;
#endif
    float rp[SRW], cp[4];
    sym_compute(raw, TI, TJ, I.n, v, rp, cp);
    const int nx = it + gridDim.x;
    if (nx < total) sym_load(I.Qp + (size_t)nx * STB * STB, raw);
    float* Ps = I.sp + (size_t)s * T * ldp;
    const float rv = warp_rows16(rp);
    if (!(lane & 1)) Ps[(size_t)TJ * ldp + (size_t)TI * STB + warp * SRW + sym_row(lane)] = rv;
    if (TI != TJ) {
      *reinterpret_cast<float4*>(sred + warp * STB + lane * 4) = make_float4(cp[0], cp[1], cp[2], cp[3]);
      __syncthreads();
      if (tid < STB) {
        float c = sred[tid];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) c += sred[w * STB + tid];
        Ps[(size_t)TI * ldp + (size_t)TJ * STB + tid] = c;
      }
      __syncthreads();     // sred is rewritten by the next tile
    }
    if (nx >= total) break;
    it = nx;
  }
}

// The solver's coupling pass on a context with packed tiles: the tile
// products of the packed incremental trial pass when the phase is one (the
// row blocks, dots and control follow in k_sym_finish), otherwise the
// row-streaming pass (tile variant 1: 4 rows x 4 chunks per warp) with each
// CTA taking the row-block items blockIdx.x, blockIdx.x + gridDim.x, ...  A
// CTA reaches the row pass's control step only in its last item (the step
// needs all other items to have arrived), and a CTA that owns no item returns
// whatever state it reads: the state a control step leaves is never a packed
// trial (only the vector kernel sets trial_ready).
template <int ST>
__global__ void __launch_bounds__(NT, 2) k_pass_sym(const Inst* __restrict__ insts, State* __restrict__ states,
                                                    Ctrl* __restrict__ ctrl, const int* __restrict__ pmap,
                                                    const float* __restrict__ XS, const float* __restrict__ VS) {
  extern __shared__ __align__(128) uint8_t dsm[];
  __shared__ double red[NWARP * NDOT];
  __shared__ int s_dec;
  __shared__ __align__(16) float sred[NWARP * STB];
  const Inst& I = insts[0];
  State& S = states[0];
  if (sym_phase(I, S)) {
    sym_tiles(I, I.dv, sred, &ctrl->err);
    return;
  }
  for (int bid = blockIdx.x; bid < I.M * I.nrb; bid += gridDim.x)
    pass_body<ST, 4, 4, 0, 0>(insts, states, ctrl, pmap, XS, VS, dsm, red, s_dec, bid);
}

// Second kernel of a packed trial pass: one CTA per row block (grid M x T)
// sums the block's slots, applies the incremental update and goes on to the
// pass's fixed-order dot reduction and control step.  Every CTA reads the
// phase before it arrives, so none can see the state the control step
// leaves; outside a packed trial all return at once.
template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_finish(const Inst* __restrict__ insts, State* __restrict__ states,
                                                   Ctrl* __restrict__ ctrl) {
  __shared__ double red[NWARP * NDOT];
  __shared__ double sh[STB];
  __shared__ int s_dec;
  const Inst& I = insts[0];
  State& S = states[0];
  if (!sym_phase(I, S)) return;
  const int T = I.tsym;
#ifdef RAPDB_CHECKED
  if (blockIdx.x >= (unsigned)(I.M * T)) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, CHK_SYM_RANGE);
    return;
  }
#endif
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  const int i = s + I.s_off;
  const float* x = I.xf[S.xcur ^ 1];
  const float* Ps = I.sp + (size_t)s * T * T * STB;
  sym_rows(I, Ps, R, i, x, I.xl[S.xcur ^ 1], I.dv, I.U[S.ucur], I.Ulo[S.ucur], I.U[S.ucur ^ 1],
           I.Ulo[S.ucur ^ 1], I.W, I.spart + (size_t)s * NDOT * T + R, sh, red);
  pass_finish(I, S, ctrl, s, i, I.spart, T, PH_TRIAL, true, x, I.dv, red, s_dec);
}

// Stand-alone packed pass (no control), in two kernels like the solver's:
// the tile products, then W = Q_i v and U = uold + W per row block with the
// block's dot partials in spart.  Arrays are (m+1, ldv) bases indexed by the
// constraint row; xl, uol, Ulo may be null.
template <int DUMMY>
__global__ void __launch_bounds__(NT, 2) k_sym_plain(const Inst* __restrict__ insts, const float* __restrict__ v,
                                                     int* err) {
  __shared__ __align__(16) float sred[NWARP * STB];
  sym_tiles(insts[0], v, sred, err);
}

template <int DUMMY>
__global__ void __launch_bounds__(NT) k_sym_rows_plain(const Inst* __restrict__ insts, const float* __restrict__ x,
                                                       const float* __restrict__ xl, const float* __restrict__ v,
                                                       const float* __restrict__ uoh, const float* __restrict__ uol,
                                                       float* __restrict__ U, float* __restrict__ Ulo,
                                                       float* __restrict__ W, double* __restrict__ spart) {
  __shared__ double red[NWARP * NDOT];
  __shared__ double sh[STB];
  const Inst& I = insts[0];
  const int T = I.tsym;
  if (blockIdx.x >= (unsigned)(I.M * T)) return;
  const int s = blockIdx.x / T, R = blockIdx.x - s * T;
  sym_rows(I, I.sp + (size_t)s * T * T * STB, R, s + I.s_off, x, xl, v, uoh, uol, U, Ulo, W,
           spart + (size_t)s * NDOT * T + R, sh, red);
}

}  // namespace rapdb_dev
