// Fine-grained iterative ILU0 (Chow & Patel) and Jacobi-iteration triangular
// solves (Anzt, Chow & Dongarra): the "Chow Patel ILU0" entry of Section 3's
// library table, decomposition and application.  Every row is independent
// inside a sweep, so each sweep is one launch over all slices of all systems
// (Batch::all_ent, one warp per 32-row slice, one lane per row) instead of
// one launch per level or colour.
//
// Both use the storage of the exact path (kernels.cuh, factor.cuh,
// sweeps.cuh): factors warp-sliced [L | U | Dinv slices], the diagonal block
// of U held only as its inverse.  Sweeps are
// synchronous: sweep t reads the iterate of sweep t-1 from one buffer and
// writes the other (lu/lu2 for the factors, y/y2 and the output/z2 for the
// triangular solves); the buffers alternate so that the last sweep lands in
// the buffer the rest of the solver reads.
#pragma once

#include "factor.cuh"
#include "sweeps.cuh"

namespace opm {

// ------------------------------------------------------------ iterative ILU0

template <typename TF>
__device__ __forceinline__ TF *factor_buf(const Sys &S, int which) {
  return static_cast<TF *>(which ? S.lu2 : S.lu);
}

// The lane's inverse diagonal block slot (entry-planar, stride 32).
template <typename TF>
__device__ __forceinline__ TF *dinv_slot(const Sys &S, TF *lu, int row) {
  return lu + S.d_off + (int64_t)kSliceVals * (row >> 5) + (row & 31);
}

// Inverts the lane's diagonal block in place (Dinv slot), flagging a
// singular pivot as the exact factorisation does.
template <typename TF>
__device__ __forceinline__ void invert_pivot(const Sys &S, TF *lu, int i) {
  TF *Dp = dinv_slot<TF>(S, lu, i);
  TF a[9], o[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) a[c] = Dp[32 * c];
  if (!inv3<TF>(a, o)) {
    atomicCAS(&S.st->error, 0, (int32_t)OPM_ERR_ZERO_PIVOT);
    atomicMin(&S.st->err_row, i);
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) Dp[32 * c] = o[c];
}

// L_ik <- L_ik inv(U_kk) for the lane's L blocks, inv(U_kk) read from D
// (same expression as the exact factorisation).
template <typename TF>
__device__ __forceinline__ void scale_l_row(const Sys &S, int sl, bool act, TF *lu, const TF *D) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const unsigned lt = lanemask_lt();
  const int len = (i < S.n) ? __ldg(S.l_rp + i + 1) - __ldg(S.l_rp + i) : 0;
  int base = (s0 < S.n) ? __ldg(S.l_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, act ? len : 0);
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (act && len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int kc = __ldg(S.l_col + base + q);
      TF *Lp = lu + 9ll * base + q;
      const TF *Dk = D + S.d_off + (int64_t)kSliceVals * (kc >> 5) + (kc & 31);
      TF a[9], d[9], l[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        a[c] = Lp[c * cnt];
        d[c] = __ldcg(Dk + 32 * c);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          l[3 * r + c] = fma(a[3 * r], d[c], fma(a[3 * r + 1], d[3 + c], a[3 * r + 2] * d[6 + c]));
#pragma unroll
      for (int c = 0; c < 9; ++c) Lp[c * cnt] = l[c];
    }
    base += __popc(m);
  }
}

// One sweep for the lane's row: Y <- A on the row's pattern; Y_ij -= X(L_ik)
// X(U_kj) for its L blocks k in ascending order (the update lists of the
// exact factorisation, so every target sees the same FMA chain in the same
// order); then L_ij = Y_ij inv(X(U_jj)) and Dinv_i = inv(Y_ii).  At the fixed
// point this is exactly the exact factorisation's arithmetic.
template <typename TF>
__device__ __forceinline__ void cp_sweep_rows(const Sys &S, int sl, int out) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const bool act = i < S.n;
  const TF *X = factor_buf<TF>(S, out ^ 1);
  TF *Y = factor_buf<TF>(S, out);
  const unsigned lt = lanemask_lt();
  copy_row_to_factors<TF>(S, sl, act, nullptr, Y);
  const int lrow = act ? __ldg(S.l_rp + i) : 0;
  const int len = act ? __ldg(S.l_rp + i + 1) - lrow : 0;
  int base = (s0 < S.n) ? __ldg(S.l_rp + s0) : 0;
  const int lenw = (i < S.n) ? len : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, lenw);
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, lenw > k);
    if (act && len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const TF *Lp = X + 9ll * base + q;
      TF l[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) l[c] = __ldg(Lp + c * cnt);
      const int u1 = __ldg(S.upd_ptr + lrow + k + 1);
      for (int u = __ldg(S.upd_ptr + lrow + k); u < u1; ++u) {
        const int64_t ds = __ldg(S.upd_dst + u), ss = __ldg(S.upd_src + u);
        TF *Ap = Y + (ds >> 6);
        const int dstr = (int)(ds & 63);
        const TF *Up = X + (ss >> 6);
        const int sstr = (int)(ss & 63);
        TF uu[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) uu[c] = __ldg(Up + c * sstr);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            TF *ap = Ap + (3 * r + c) * dstr;
            *ap = fma(-l[3 * r], uu[c], fma(-l[3 * r + 1], uu[3 + c], fma(-l[3 * r + 2], uu[6 + c], *ap)));
          }
      }
    }
    base += __popc(m);
  }
  scale_l_row<TF>(S, sl, act, Y, X);
  if (act) invert_pivot<TF>(S, Y, i);
}

// Initial guess into buffer `out`: stage 0 copies A (from the caller's
// values when given) and inverts the diagonal blocks; stage 1 forms
// L_ij = A_ij inv(A_jj).  U_ij = A_ij needs no work.
template <typename TF>
__global__ void __launch_bounds__(256) k_cp_init(Batch B, int stage, int out) {
  pdl_enter();
  const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= B.nall) return;
  const int4 E = B.all_ent[e];
  const Sys &S = B.sys[E.x];
  if (S.skip) return;
  const int i = E.y * 32 + (threadIdx.x & 31);
  const bool act = i < S.n;
  TF *Y = factor_buf<TF>(S, out);
  if (stage == 0) {
    copy_row_to_factors<TF>(S, E.y, act, S.vals_in, Y);
    if (act) invert_pivot<TF>(S, Y, i);
  } else {
    scale_l_row<TF>(S, E.y, act, Y, Y);
  }
}

// One synchronous sweep: reads buffer out^1, writes buffer out.
template <typename TF>
__global__ void __launch_bounds__(256) k_cp_sweep(Batch B, int out) {
  pdl_enter();
  const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= B.nall) return;
  const int4 E = B.all_ent[e];
  if (B.sys[E.x].skip) return;
  cp_sweep_rows<TF>(B.sys[E.x], E.y, out);
}

// ------------------------------------------------------ Jacobi triangular solves

// The right-hand side of the preconditioner application (equation 3's r):
// h = r + beta (p - omega v) for MODE P, r - alpha v for MODE S, stored to p
// or s as the exact forward sweep does.  MODE plain reads w as is.
template <int MODE>
__global__ void __launch_bounds__(256, 6) k_jac_rhs(Batch B) {
  pdl_enter();
  OPM_TILE(B, S, lt);
  const DevState *st = S.st;
  if (!running(st)) return;
  const double c1 = (MODE == kModeP) ? st->beta : st->alpha;
  const double c2 = (MODE == kModeP) ? st->omega : 0.0;
  double *hout = (MODE == kModeP) ? S.p : S.s;
  OPM_TILE_ROWS(i, lt) {
    if (i < S.n) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int64_t q = 3ll * i + c;
        const double rr = S.r[q], vo = S.v[q];
        hout[q] = (MODE == kModeP) ? fma(c1, fma(-c2, vo, hout[q]), rr) : fma(-c1, vo, rr);
      }
    }
  }
}

template <int MODE>
__device__ __forceinline__ const double *jac_rhs(const Sys &S) {
  return (MODE == kModePlain) ? S.w : (MODE == kModeP) ? S.p : S.s;
}

// Forward iterate t (1-based) lives in y for odd t, y2 for even t.
template <typename TF>
__device__ __forceinline__ TF *jac_y(const Sys &S, int t) {
  return static_cast<TF *>((t & 1) ? S.y : S.y2);
}

// Backward iterate t (0-based) of T: the last one lands in the sweep output.
template <int MODE>
__device__ __forceinline__ double *jac_z(const Sys &S, int t, int T) {
  return ((T - t) & 1) ? S.z2 : sweep_out<MODE>(S);
}

// Forward sweep t of T: y_t = h - L y_{t-1} with y_0 = h.  The last sweep
// also starts the backward iteration, z_0 = inv(U_ii) y_T.
template <typename TF, int MODE>
__global__ void __launch_bounds__(256, 4) k_jac_fwd(Batch B, int t, int T) {
  pdl_enter();
  const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= B.nall) return;
  const int4 E = B.all_ent[e];
  const Sys &S = B.sys[E.x];
  if (MODE != kModePlain && !running(S.st)) return;
  const int lane = threadIdx.x & 31;
  const int s0 = E.y * 32;
  const int i = s0 + lane;
  const bool act = i < S.n;
  const TF *lu = static_cast<const TF *>(S.lu);
  const double *h = jac_rhs<MODE>(S);
  const int len = act ? __ldg(S.l_rp + i + 1) - __ldg(S.l_rp + i) : 0;
  const int base = (s0 < S.n) ? __ldg(S.l_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  TF a0 = TF(0), a1 = TF(0), a2 = TF(0);
  if (act) {
    const Vec3<double> hi = load3cg(h + 3ll * i);
    a0 = (TF)hi.c0;
    a1 = (TF)hi.c1;
    a2 = (TF)hi.c2;
  }
  if (t == 1) row_sub<TF, double>(S.l_col, lu, h, len, base, 0, maxlen, act, a0, a1, a2);
  else row_sub<TF, TF>(S.l_col, lu, jac_y<TF>(S, t - 1), len, base, 0, maxlen, act, a0, a1, a2);
  if (act) {
    TF *yo = jac_y<TF>(S, t) + 3ll * i;
    yo[0] = a0;
    yo[1] = a1;
    yo[2] = a2;
    if (t == T) {
      TF d[9];
      load_dinv<TF>(lu + S.d_off + (int64_t)kSliceVals * E.y + lane, d);
      store_dinv_product<TF>(jac_z<MODE>(S, 0, T) + 3ll * i, d, a0, a1, a2);
    }
  }
}

// Backward sweep t of T: z_t = inv(U_ii)(y_T - U_off z_{t-1}).
template <typename TF, int MODE>
__global__ void __launch_bounds__(256, 4) k_jac_bwd(Batch B, int t, int T) {
  pdl_enter();
  const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= B.nall) return;
  const int4 E = B.all_ent[e];
  const Sys &S = B.sys[E.x];
  if (MODE != kModePlain && !running(S.st)) return;
  const int lane = threadIdx.x & 31;
  const int s0 = E.y * 32;
  const int i = s0 + lane;
  const bool act = i < S.n;
  const TF *lu = static_cast<const TF *>(S.lu);
  const int len = act ? __ldg(S.u_rp + i + 1) - __ldg(S.u_rp + i) : 0;
  const int base = (s0 < S.n) ? __ldg(S.u_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  TF a0 = TF(0), a1 = TF(0), a2 = TF(0);
  if (act) {
    const Vec3<TF> yi = load3cg(jac_y<TF>(S, T) + 3ll * i);
    a0 = yi.c0;
    a1 = yi.c1;
    a2 = yi.c2;
  }
  row_sub<TF, double>(S.u_col, lu + S.u_off, jac_z<MODE>(S, t - 1, T), len, base, 0, maxlen, act, a0, a1, a2);
  if (act) {
    TF d[9];
    load_dinv<TF>(lu + S.d_off + (int64_t)kSliceVals * E.y + lane, d);
    store_dinv_product<TF>(jac_z<MODE>(S, t, T) + 3ll * i, d, a0, a1, a2);
  }
}

}  // namespace opm
