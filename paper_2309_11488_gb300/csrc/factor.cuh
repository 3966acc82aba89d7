// ILU0 decomposition (Algorithm 2) on sm_103a, fused with the value
// permutation (Algorithm 3's copy): phase by phase, one warp per 32-row slice
// and one lane per row, the row's eliminations in the order of its L blocks.
#pragma once

#include "kernels.cuh"

namespace opm {

// Copies the lane's row of A into its L / D / U slots of the factor buffer
// lu (the diagonal block into the Dinv slot, inverted later).  With
// vals_user, block w of the permuted matrix comes from the caller's block
// a_src[w] (Algorithm 3's index copy) and is also stored into A; without, A
// is read.  Blocks outside the preconditioner's pattern have no slot.
template <typename TF>
__device__ __forceinline__ void copy_row_to_factors(const Sys &S, int sl, bool act, const double *vals_user,
                                                    TF *lu) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const unsigned lt = lanemask_lt();
  const int len = (i < n) ? __ldg(S.a_rp + i + 1) - __ldg(S.a_rp + i) : 0;
  int base = (s0 < n) ? __ldg(S.a_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, act ? len : 0);
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (act && len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int w = base + q;
      const int64_t dst = __ldg(S.a_dst + w);
      const int64_t doff = dst >> 6;
      const int dstr = (int)(dst & 63);
      double *av = S.a_val + 9ll * base + q;
      double e[9];
      if (vals_user) {
        // the permuted copy is next read by the SpMV: its stores are marked
        // evict-first, which keeps the pivot rows' inverses and U blocks in
        // L2 for the gathers
        const double *src = vals_user + 9ll * __ldg(S.a_src + w);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          e[c] = __ldg(src + c);
          __stcs(av + c * cnt, e[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) e[c] = av[c * cnt];
      }
      if (dst >= 0) {
#pragma unroll
        for (int c = 0; c < 9; ++c) lu[doff + (int64_t)c * dstr] = (TF)e[c];
      }
    }
    base += __popc(m);
  }
}

// ILU0 decomposition (Algorithm 2) of the permuted matrix, phase by phase,
// fused with the value permutation: with vals_in, block w of the permuted
// matrix is copied from the caller's block a_src[w] (Algorithm 3's index
// copy) into both A and the factors.  Row i of a phase reads only rows of
// earlier phases (its pivots k < i) and updates only its own blocks.
template <typename TF>
__device__ __forceinline__ void factor_rows(const Sys &S, int sl, int r0, int r1) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const bool act = i >= r0 && i < r1;
  TF *lu = static_cast<TF *>(S.lu);
  const double *__restrict__ vals_user = S.vals_in;
  const unsigned lt = lanemask_lt();
  DevState *st = S.st;
  copy_row_to_factors<TF>(S, sl, act, vals_user, lu);
  // ---- eliminate with the pivots k < i (Algorithm 2's updates of row i)
  const int lrow = (i < n) ? __ldg(S.l_rp + i) : 0;
  const int len = (i < n) ? __ldg(S.l_rp + i + 1) - lrow : 0;
  int base = (s0 < n) ? __ldg(S.l_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, act ? len : 0);
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (act && len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int kc = __ldg(S.l_col + base + q);
      TF *Lp = lu + 9ll * base + q;
      const TF *Dk = lu + S.d_off + (int64_t)kSliceVals * (kc >> 5) + (kc & 31);
      TF a[9], d[9], l[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        a[c] = Lp[c * cnt];
        d[c] = __ldcg(Dk + 32 * c);
      }
      // L_ik = A_ik * inv(U_kk)
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          l[3 * r + c] = fma(a[3 * r], d[c], fma(a[3 * r + 1], d[3 + c], a[3 * r + 2] * d[6 + c]));
#pragma unroll
      for (int c = 0; c < 9; ++c) Lp[c * cnt] = l[c];
      // A_ij -= L_ik * U_kj for the listed j
      const int u1 = __ldg(S.upd_ptr + lrow + k + 1);
      for (int u = __ldg(S.upd_ptr + lrow + k); u < u1; ++u) {
        const int64_t ds = __ldg(S.upd_dst + u), ss = __ldg(S.upd_src + u);
        TF *Ap = lu + (ds >> 6);
        const int dstr = (int)(ds & 63);
        const TF *Up = lu + (ss >> 6);
        const int sstr = (int)(ss & 63);
        TF uu[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) uu[c] = __ldcg(Up + c * sstr);
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
  if (act) {
    TF *Dp = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
    TF a[9], o[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) a[c] = Dp[32 * c];
    if (!inv3<TF>(a, o)) {
      atomicCAS(&st->error, 0, (int32_t)OPM_ERR_ZERO_PIVOT);
      atomicMin(&st->err_row, i);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) Dp[32 * c] = o[c];
  }
}

template <typename TF>
__global__ void __launch_bounds__(256) k_factor_phase(Batch B, int c) {
  pdl_enter();
  const int e = __ldg(B.fwd_ptr + c) + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= __ldg(B.fwd_ptr + c + 1)) return;
  const int4 E = B.ent[e];
  factor_rows<TF>(B.sys[E.x], E.y, E.z, E.w);
}

template <typename TF>
__global__ void __launch_bounds__(1024) k_factor(Batch B) {
  const int W = gridDim.x * (blockDim.x >> 5);
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  bool timed_out = false;
  for (int c = 0; c < B.nphases; ++c) {
    if (c > 0) grid_sync(B, timed_out);
    const int e1 = __ldg(B.fwd_ptr + c + 1);
    for (int e = __ldg(B.fwd_ptr + c) + g; e < e1; e += W) {
      const int4 E = B.ent[e];
      factor_rows<TF>(B.sys[E.x], E.y, E.z, E.w);
    }
  }
}

}  // namespace opm
