// ILU0 application (Algorithm 1) on sm_103a: forward and backward block
// substitution over the schedule's phases, one warp per 32-row slice and one
// lane per row of the warp-sliced factors, fused with the BiCGStab update
// that forms the right-hand side.  Two launch forms per phase (throughput and
// latency) and one cooperative form walking every phase.
//
// Values produced in earlier phases by other SMs are read through L2
// (ld.global.cg), never from L1.
#pragma once

#include "kernels.cuh"

namespace opm {

template <typename TF>
struct Vec3 {
  TF c0, c1, c2;
};

template <typename TF>
__device__ __forceinline__ Vec3<TF> load3cg(const TF *p) {
  return {__ldcg(p), __ldcg(p + 1), __ldcg(p + 2)};
}

// a -= B v for one 3x3 block held in registers, in FMA form.  Every sweep
// path goes through this one expression, so all of them round alike.
template <typename TF>
__device__ __forceinline__ void blk_sub_r(const TF (&b)[9], TF v0, TF v1, TF v2, TF &a0, TF &a1, TF &a2) {
  a0 = fma(-b[0], v0, fma(-b[1], v1, fma(-b[2], v2, a0)));
  a1 = fma(-b[3], v0, fma(-b[4], v1, fma(-b[5], v2, a1)));
  a2 = fma(-b[6], v0, fma(-b[7], v1, fma(-b[8], v2, a2)));
}

// The same for a block in memory, entry-planar with stride c.  Factor
// values and their column indices are read once per application: streaming
// loads (evict-first in L1 and L2) leave the cache to the vectors that the
// next kernels read again.
template <typename TF>
__device__ __forceinline__ void blk_sub(const TF *__restrict__ Bv, int c, TF v0, TF v1, TF v2, TF &a0, TF &a1,
                                        TF &a2) {
  TF b[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) b[e] = __ldcs(Bv + e * c);
  blk_sub_r<TF>(b, v0, v1, v2, a0, a1, a2);
}

// a -= sum over the lane's row of a sliced part of B_ij v_j for the slabs
// k0, k0+1, ... (base = first block of slab k0), v read through L2; two
// slabs per step for memory-level parallelism.  All lanes call with len =
// their row's block count (0 past n), which defines the slab layout of the
// slice; lanes with !act issue no loads.
template <typename TF, typename TV>
__device__ __forceinline__ void row_sub(const int32_t *__restrict__ col, const TF *__restrict__ vals,
                                        const TV *vec, int len, int base, int k0, int maxlen, bool act, TF &a0,
                                        TF &a1, TF &a2) {
  const unsigned lt = lanemask_lt();
  for (int k = k0; k < maxlen; k += 2) {
    const unsigned m0 = __ballot_sync(0xffffffffu, len > k);
    const unsigned m1 = __ballot_sync(0xffffffffu, len > k + 1);
    const int b0 = base, b1 = base + __popc(m0);
    base = b1 + __popc(m1);
    const bool u0 = act && len > k, u1 = act && len > k + 1;
    const int q0 = __popc(m0 & lt), q1 = __popc(m1 & lt);
    int j0 = 0, j1 = 0;
    if (u0) j0 = __ldcs(col + b0 + q0);
    if (u1) j1 = __ldcs(col + b1 + q1);
    if (u0) {
      const Vec3<TV> v = load3cg(vec + 3ll * j0);
      blk_sub<TF>(vals + 9ll * b0 + q0, __popc(m0), (TF)v.c0, (TF)v.c1, (TF)v.c2, a0, a1, a2);
    }
    if (u1) {
      const Vec3<TV> v = load3cg(vec + 3ll * j1);
      blk_sub<TF>(vals + 9ll * b1 + q1, __popc(m1), (TF)v.c0, (TF)v.c1, (TF)v.c2, a0, a1, a2);
    }
  }
}

// The first PRE slabs of the lane's row, loaded ahead: column, block values.
// Returns the first block of slab PRE.
template <typename TF, int PRE>
__device__ __forceinline__ int preload_slabs(const int32_t *__restrict__ col, const TF *__restrict__ vals, int len,
                                             int base, bool act, int (&jp)[PRE], TF (&bp)[PRE][9]) {
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < PRE; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (act && len > k) {
      const int q = __popc(m & lt), cnt = __popc(m);
      jp[k] = __ldcs(col + base + q);
#pragma unroll
      for (int e = 0; e < 9; ++e) bp[k][e] = __ldcs(vals + 9ll * base + q + e * cnt);
    }
    base += __popc(m);
  }
  return base;
}

// Gathers of the preloaded slabs' vector blocks (issued together).
template <typename TV, int PRE>
__device__ __forceinline__ void gather_preloaded(const TV *vec, int len, bool act, const int (&jp)[PRE],
                                                 Vec3<TV> (&vv)[PRE]) {
#pragma unroll
  for (int k = 0; k < PRE; ++k)
    if (act && len > k) vv[k] = load3cg(vec + 3ll * jp[k]);
}

// a -= B_k v_k over the preloaded slabs, in slab order.
template <typename TF, typename TV, int PRE>
__device__ __forceinline__ void preloaded_sub(int len, bool act, const TF (&bp)[PRE][9], const Vec3<TV> (&vv)[PRE],
                                              TF &a0, TF &a1, TF &a2) {
#pragma unroll
  for (int k = 0; k < PRE; ++k)
    if (act && len > k) blk_sub_r<TF>(bp[k], (TF)vv[k].c0, (TF)vv[k].c1, (TF)vv[k].c2, a0, a1, a2);
}

// z_i = inv(U_ii) a with the inverse diagonal block (entry-planar, stride 32).
template <typename TF>
__device__ __forceinline__ void load_dinv(const TF *D, TF (&d)[9]) {
#pragma unroll
  for (int e = 0; e < 9; ++e) d[e] = __ldcs(D + 32 * e);
}

template <typename TF>
__device__ __forceinline__ void store_dinv_product(double *zi, const TF (&d)[9], TF a0, TF a1, TF a2) {
  zi[0] = (double)fma(d[0], a0, fma(d[1], a1, d[2] * a2));
  zi[1] = (double)fma(d[3], a0, fma(d[4], a1, d[5] * a2));
  zi[2] = (double)fma(d[6], a0, fma(d[7], a1, d[8] * a2));
}

template <int MODE>
__device__ __forceinline__ double *sweep_out(const Sys &S) {
  return (MODE == kModeP) ? S.ph : (MODE == kModeS) ? S.sh : S.t;
}

// Forward substitution for the rows of slice sl inside [r0, r1):
// y_i = rhs_i - sum_{j<i} L_ij y_j (Algorithm 1, equation 3), the right-hand
// side formed on the fly.  A row without U blocks takes its backward step
// z_i = inv(U_ii) y_i (equation 4) at once; y_i is stored only when a later
// step reads it.
//
// PRE > 0 is the latency-oriented form for small phases: the row's constant
// data (lengths, first PRE slabs, inverse diagonal) is loaded before the
// wait for the preceding kernel (programmatic dependent launch), so only the
// gathers of earlier phases' results remain after it.  PRE == 0 expects the
// caller to have waited.  Both forms do the same arithmetic in the same order.
template <typename TF, int MODE, int PRE>
__device__ __forceinline__ void fwd_rows(const Sys &S, int sl, int r0, int r1) {
  constexpr int NP = PRE > 0 ? PRE : 1;
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const bool act = i >= r0 && i < r1;
  // constant for the whole solve: safe to read before the wait
  TF *y = static_cast<TF *>(S.y);
  const TF *lu = static_cast<const TF *>(S.lu);
  const DevState *st = S.st;
  const double *rin = (MODE == kModePlain) ? S.w : S.r;
  const double *vin = S.v;
  double *hout = (MODE == kModeP) ? S.p : S.s;
  double *zout = sweep_out<MODE>(S);
  const uint2 M = __ldg(S.sl_mask + sl);
  const bool eager = (M.x >> lane) & 1u, ystore = (M.y >> lane) & 1u;
  const int len = (i < S.n) ? __ldg(S.l_rp + i + 1) - __ldg(S.l_rp + i) : 0;
  int base = (s0 < S.n) ? __ldg(S.l_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  const TF *D = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
  int jp[NP];
  TF bp[NP][9], d[9];
  Vec3<TF> vv[NP];
  if (PRE > 0) {
    base = preload_slabs<TF, NP>(S.l_col, lu, len, base, act, jp, bp);
    if (act && eager) load_dinv<TF>(D, d);
    pdl_wait();
  }
  // after the wait: the solver state, the right-hand side and the results
  // of earlier phases, all issued before the first use
  const int status = st->status, err = st->error;
  const double c1 = (MODE == kModeP) ? st->beta : (MODE == kModeS) ? st->alpha : 0.0;
  const double c2 = (MODE == kModeP) ? st->omega : 0.0;
  Vec3<double> rr{0.0, 0.0, 0.0}, vo{0.0, 0.0, 0.0}, po{0.0, 0.0, 0.0};
  if (act) {
    rr = load3cg(rin + 3ll * i);
    if (MODE != kModePlain) vo = load3cg(vin + 3ll * i);
    if (MODE == kModeP) po = load3cg(hout + 3ll * i);
  }
  if (PRE > 0) gather_preloaded<TF, NP>(y, len, act, jp, vv);
  if (MODE != kModePlain && !(status == kRunning && err == 0)) return;
  double h0 = rr.c0, h1 = rr.c1, h2 = rr.c2;
  if (act) {
    if (MODE == kModeP) {
      h0 = fma(c1, fma(-c2, vo.c0, po.c0), rr.c0);
      h1 = fma(c1, fma(-c2, vo.c1, po.c1), rr.c1);
      h2 = fma(c1, fma(-c2, vo.c2, po.c2), rr.c2);
    } else if (MODE == kModeS) {
      h0 = fma(-c1, vo.c0, rr.c0);
      h1 = fma(-c1, vo.c1, rr.c1);
      h2 = fma(-c1, vo.c2, rr.c2);
    }
    if (MODE != kModePlain) {
      double *ho = hout + 3ll * i;
      ho[0] = h0; ho[1] = h1; ho[2] = h2;
    }
  }
  TF a0 = (TF)h0, a1 = (TF)h1, a2 = (TF)h2;
  if (PRE > 0) preloaded_sub<TF, TF, NP>(len, act, bp, vv, a0, a1, a2);
  row_sub<TF, TF>(S.l_col, lu, y, len, base, PRE, maxlen, act, a0, a1, a2);
  if (act) {
    if (eager) {
      if (PRE == 0) load_dinv<TF>(D, d);
      store_dinv_product<TF>(zout + 3ll * i, d, a0, a1, a2);
    }
    if (ystore) {
      TF *yi = y + 3ll * i;
      yi[0] = a0; yi[1] = a1; yi[2] = a2;
    }
  }
}

// Backward substitution for the rows of slice sl inside [r0, r1) that have
// U blocks: z_i = inv(U_ii)(y_i - sum_{j>i} U_ij z_j) (Algorithm 1,
// equation 4).  PRE as for fwd_rows.  With FP64 factors, the rows whose
// product after the application takes the upper sum w_i = sum_{j>i} U_ij z_j
// (sp_mask.y) store it in uz as y_i - a, a = y_i - sum_{j>i} U_ij z_j being
// the walk's result (y_i read again: it is not kept live across the walk).
template <typename TF, int MODE, int PRE>
__device__ __forceinline__ void bwd_rows(const Sys &S, int sl, int r0, int r1) {
  constexpr int NP = PRE > 0 ? PRE : 1;
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const uint2 M = __ldg(S.sl_mask + sl);
  const bool act = i >= r0 && i < r1 && !((M.x >> lane) & 1u);
  const TF *y = static_cast<const TF *>(S.y);
  const TF *lu = static_cast<const TF *>(S.lu);
  const DevState *st = S.st;
  double *z = sweep_out<MODE>(S);
  const int len = (i < S.n) ? __ldg(S.u_rp + i + 1) - __ldg(S.u_rp + i) : 0;
  int base = (s0 < S.n) ? __ldg(S.u_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  const TF *D = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
  int jp[NP];
  TF bp[NP][9], d[9];
  Vec3<double> vv[NP];
  if (PRE > 0) {
    base = preload_slabs<TF, NP>(S.u_col, lu + S.u_off, len, base, act, jp, bp);
    if (act) load_dinv<TF>(D, d);
    pdl_wait();
  }
  const int status = st->status, err = st->error;
  Vec3<TF> yi{TF(0), TF(0), TF(0)};
  if (act) yi = load3cg(y + 3ll * i);
  if (PRE > 0) gather_preloaded<double, NP>(z, len, act, jp, vv);
  if (MODE != kModePlain && !(status == kRunning && err == 0)) return;
  TF a0 = yi.c0, a1 = yi.c1, a2 = yi.c2;
  if (PRE > 0) preloaded_sub<TF, double, NP>(len, act, bp, vv, a0, a1, a2);
  row_sub<TF, double>(S.u_col, lu + S.u_off, z, len, base, PRE, maxlen, act, a0, a1, a2);
  if (act) {
    if (sizeof(TF) == sizeof(double) && S.uz && ((__ldg(S.sp_mask + sl).y >> lane) & 1u)) {
      const Vec3<TF> yr = load3cg(y + 3ll * i);
      double *w = S.uz + 3ll * i;
      w[0] = (double)(yr.c0 - a0);
      w[1] = (double)(yr.c1 - a1);
      w[2] = (double)(yr.c2 - a2);
    }
    if (PRE == 0) load_dinv<TF>(D, d);
    store_dinv_product<TF>(z + 3ll * i, d, a0, a1, a2);
  }
}

// The forward step of the first phase, whose rows have no L blocks (no
// earlier row precedes them): y_i = rhs_i, z_i = inv(U_ii) y_i for rows
// without U blocks.  The same expressions as fwd_rows, without its walk of
// the L blocks, and with the register budget of a streaming kernel (eight
// CTAs per SM) so that the many short warps overlap their few loads.
template <typename TF, int MODE>
__global__ void __launch_bounds__(256, 8) k_fwd_first(Batch B) {
  pdl_trigger();
  const int e = __ldg(B.fwd_ptr) + blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= __ldg(B.fwd_ptr + 1)) return;
  const int4 E = B.ent[e];
  const Sys &S = B.sys[E.x];
  const int lane = threadIdx.x & 31;
  const int i = E.y * 32 + lane;
  if (i < E.z || i >= E.w) return;
  const uint2 M = __ldg(S.sl_mask + E.y);
  const bool eager = (M.x >> lane) & 1u, ystore = (M.y >> lane) & 1u;
  pdl_wait();
  const DevState *st = S.st;
  if (MODE != kModePlain && !running(st)) return;
  const double *rin = (MODE == kModePlain) ? S.w : S.r;
  double *hout = (MODE == kModeP) ? S.p : S.s;
  const Vec3<double> rr = load3cg(rin + 3ll * i);
  double h0 = rr.c0, h1 = rr.c1, h2 = rr.c2;
  if (MODE != kModePlain) {
    const Vec3<double> vo = load3cg(S.v + 3ll * i);
    if (MODE == kModeP) {
      const double c1 = st->beta, c2 = st->omega;
      const Vec3<double> po = load3cg(hout + 3ll * i);
      h0 = fma(c1, fma(-c2, vo.c0, po.c0), rr.c0);
      h1 = fma(c1, fma(-c2, vo.c1, po.c1), rr.c1);
      h2 = fma(c1, fma(-c2, vo.c2, po.c2), rr.c2);
    } else {
      const double c1 = st->alpha;
      h0 = fma(-c1, vo.c0, rr.c0);
      h1 = fma(-c1, vo.c1, rr.c1);
      h2 = fma(-c1, vo.c2, rr.c2);
    }
    double *ho = hout + 3ll * i;
    ho[0] = h0; ho[1] = h1; ho[2] = h2;
  }
  const TF a0 = (TF)h0, a1 = (TF)h1, a2 = (TF)h2;
  if (eager) {
    TF d[9];
    load_dinv<TF>(static_cast<const TF *>(S.lu) + S.d_off + (int64_t)kSliceVals * E.y + lane, d);
    store_dinv_product<TF>(sweep_out<MODE>(S) + 3ll * i, d, a0, a1, a2);
  }
  if (ystore) {
    TF *yi = static_cast<TF *>(S.y) + 3ll * i;
    yi[0] = a0; yi[1] = a1; yi[2] = a2;
  }
}

// One launch per phase, one sweep entry (a 32-row slice) per warp.  PRE = 0:
// throughput form for large phases (256 threads); PRE > 0: latency form for
// small phases (64 threads, so the few warps spread over all SMs).
template <typename TF, int MODE, int PRE>
__global__ void __launch_bounds__(PRE > 0 ? 64 : 256, PRE > 0 ? 1 : 4) k_fwd_phase(Batch B, int c) {
  pdl_trigger();
  if (PRE == 0) pdl_wait();
  const int e = __ldg(B.fwd_ptr + c) + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= __ldg(B.fwd_ptr + c + 1)) return;
  const int4 E = B.ent[e];
  fwd_rows<TF, MODE, PRE>(B.sys[E.x], E.y, E.z, E.w);
}

template <typename TF, int MODE, int PRE>
__global__ void __launch_bounds__(PRE > 0 ? 64 : 256, PRE > 0 ? 1 : 4) k_bwd_phase(Batch B, int c) {
  pdl_trigger();
  if (PRE == 0) pdl_wait();
  const int e = __ldg(B.bwd_ptr + c) + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= __ldg(B.bwd_ptr + c + 1)) return;
  const int4 E = B.ent[e];
  bwd_rows<TF, MODE, PRE>(B.sys[E.x], E.y, E.z, E.w);
}

// ILU0 application z = U^-1 L^-1 rhs (Algorithm 1) in one cooperative
// launch: forward phases in order, then backward phases in reverse order.
template <typename TF, int MODE>
__global__ void __launch_bounds__(1024) k_apply(Batch B) {
  const int W = gridDim.x * (blockDim.x >> 5);
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  bool timed_out = false;
  for (int c = 0; c < B.nphases; ++c) {
    if (c > 0) grid_sync(B, timed_out);
    const int e1 = __ldg(B.fwd_ptr + c + 1);
    for (int e = __ldg(B.fwd_ptr + c) + g; e < e1; e += W) {
      const int4 E = B.ent[e];
      fwd_rows<TF, MODE, 0>(B.sys[E.x], E.y, E.z, E.w);
    }
  }
  for (int c = B.nphases - 1; c >= 0; --c) {
    const int e0 = __ldg(B.bwd_ptr + c), e1 = __ldg(B.bwd_ptr + c + 1);
    if (e0 == e1) continue;  // uniform over the grid: every CTA skips together
    grid_sync(B, timed_out);
    for (int e = e0 + g; e < e1; e += W) {
      const int4 E = B.ent[e];
      bwd_rows<TF, MODE, 0>(B.sys[E.x], E.y, E.z, E.w);
    }
  }
}

}  // namespace opm
