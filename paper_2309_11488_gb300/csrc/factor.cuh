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

// One-pass rows (every update of the row is A_ii -= L_ik U_ki, Algorithm 2
// restricted to this pattern): the lane walks its row once in A's order --
// the diagonal first, kept in registers, then L blocks in column order, then
// U blocks -- copying each block from the caller (Algorithm 3's index copy)
// into A and into its factor slot; an L block becomes L_ik = A_ik inv(U_kk)
// and at once updates the diagonal with the U_ki its a_aux names.  The same
// expressions, in the same order, as the general path below, so both paths
// give the same bits.  Loads of a block (its indices, the caller's values,
// the pivot's inverse and U_ki) do not wait for the previous block's stores.
// With DREG false the diagonal stays in its factor slot (read-modify-write
// per update, as the two-step path does) instead of registers: fewer
// registers, the same expressions.
template <typename TF, bool DREG>
__device__ __forceinline__ void one_pass_rows(const Sys &S, int sl, bool fz, const double *__restrict__ vals_user,
                                              TF *lu, TF (&D)[9]) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const unsigned lt = lanemask_lt();
  const int len = (i < n) ? __ldg(S.a_rp + i + 1) - __ldg(S.a_rp + i) : 0;
  int base = (s0 < n) ? __ldg(S.a_rp + s0) : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, fz ? len : 0);
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (fz && len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int w = base + q;
      const int64_t dst = __ldg(S.a_dst + w);
      const int col = __ldg(S.a_col + w);
      const int64_t aux = __ldg(S.a_aux + w);
      double *av = S.a_val + 9ll * base + q;
      double e[9];
      if (vals_user) {
        const double *src = vals_user + 9ll * __ldg(S.a_src + w);
#pragma unroll
        for (int c = 0; c < 9; ++c) e[c] = __ldg(src + c);
#pragma unroll
        for (int c = 0; c < 9; ++c) __stcs(av + c * cnt, e[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) e[c] = av[c * cnt];
      }
      const int64_t doff = dst >> 6;
      const int dstr = (int)(dst & 63);
      TF *Dp = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
      if (k == 0) {
        if (DREG) {
#pragma unroll
          for (int c = 0; c < 9; ++c) D[c] = (TF)e[c];
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) Dp[32 * c] = (TF)e[c];
        }
      } else if (col < i && dst >= 0) {
        const TF *Dk = lu + S.d_off + (int64_t)kSliceVals * (col >> 5) + (col & 31);
        TF d[9], l[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) d[c] = __ldcg(Dk + 32 * c);
        // L_ik = A_ik * inv(U_kk)
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            l[3 * r + c] = fma((TF)e[3 * r], d[c], fma((TF)e[3 * r + 1], d[3 + c], (TF)e[3 * r + 2] * d[6 + c]));
#pragma unroll
        for (int c = 0; c < 9; ++c) lu[doff + (int64_t)c * dstr] = l[c];
        if (aux >= 0) {
          const TF *Up = lu + (aux >> 6);
          const int sstr = (int)(aux & 63);
          TF uu[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) uu[c] = __ldcg(Up + c * sstr);
          // A_ii -= L_ik * U_ki
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              TF &dv = DREG ? D[3 * r + c] : Dp[32 * (3 * r + c)];
              dv = fma(-l[3 * r], uu[c], fma(-l[3 * r + 1], uu[3 + c], fma(-l[3 * r + 2], uu[6 + c], dv)));
            }
        }
      } else if (dst >= 0) {
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
// With ONE_PASS, one-pass rows take one_pass_rows; the others (all rows
// without ONE_PASS: the cooperative kernel, whose register budget is that of
// 1024-thread CTAs) copy their row first and then eliminate with the update
// lists.
// With EARLY_COPY (a kernel launched as a programmatic dependent that has
// not waited yet) the two-step path copies its rows before pdl_wait: the
// copy reads only the caller's values and writes only the phase's own rows,
// so it overlaps the tail of the previous phase; the elimination, which
// reads earlier phases' pivots, comes after the wait.
template <typename TF, bool ONE_PASS, bool EARLY_COPY = false, bool DREG = true>
__device__ __forceinline__ void factor_rows(const Sys &S, int sl, int r0, int r1) {
  if (S.skip) return;  // warp-uniform: the entry belongs to one system
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const bool act = i >= r0 && i < r1;
  const bool fz = ONE_PASS && act && ((__ldg(S.fz_mask + sl) >> lane) & 1u);
  const bool gen = act && !fz;
  TF *lu = static_cast<TF *>(S.lu);
  const double *__restrict__ vals_user = S.vals_in;
  const unsigned lt = lanemask_lt();
  DevState *st = S.st;
  TF D[9];
  if (ONE_PASS && __any_sync(0xffffffffu, fz)) one_pass_rows<TF, DREG>(S, sl, fz, vals_user, lu, D);
  if (__any_sync(0xffffffffu, gen)) {
    copy_row_to_factors<TF>(S, sl, gen, vals_user, lu);
    if (EARLY_COPY) pdl_wait();
    // ---- eliminate with the pivots k < i (Algorithm 2's updates of row i)
    const int lrow = (i < n) ? __ldg(S.l_rp + i) : 0;
    const int len = (i < n) ? __ldg(S.l_rp + i + 1) - lrow : 0;
    int base = (s0 < n) ? __ldg(S.l_rp + s0) : 0;
    const int maxlen = __reduce_max_sync(0xffffffffu, gen ? len : 0);
    for (int k = 0; k < maxlen; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, len > k);
      if (gen && len > k) {
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
  }
  if (act) {
    TF *Dp = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
    TF a[9], o[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) a[c] = (fz && DREG) ? D[c] : Dp[32 * c];
    if (!inv3<TF>(a, o)) {
      atomicCAS(&st->error, 0, (int32_t)OPM_ERR_ZERO_PIVOT);
      atomicMin(&st->err_row, i);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) Dp[32 * c] = o[c];
  }
}

// One launch per phase, one 32-row slice per warp.  ONE_PASS takes the
// one-pass walk for the rows that allow it, DREG keeps its diagonal in
// registers; MINB is the launch's resident CTAs per SM.  Measured at the
// 949,871-cell workload (event-timed refactorisations, A/B in one process):
// FP32 factors 0.509 -> 0.460 ms with the one-pass walk (diagonal in
// registers) at four CTAs per SM.  FP64 factors are bound by the FP64 pipe
// in the large phases (54 FMAs per L block): with the diagonal in registers
// (104 registers) the walk lost more occupancy than its shorter load chains
// gained (0.685 -> 0.696 ms at three CTAs per SM); with the diagonal in its
// slot (64 registers, four CTAs per SM) it gains 0.668 -> 0.655 ms over the
// two-step path.  The small phases, latency chains, keep the two-step path
// for FP64 (the walk's registers made them slower: 0.668 -> 0.694 ms); the
// two-step path copies before the dependency wait (0.705 -> 0.694 ms).
template <typename TF, bool ONE_PASS, int MINB, bool DREG = true>
__global__ void __launch_bounds__(256, MINB) k_factor_phase(Batch B, int c) {
  // the two-step path waits after its copy (EARLY_COPY); the one-pass walk
  // needs earlier phases from its first L block on
  if (ONE_PASS) pdl_enter();
  else pdl_trigger();
  const int e = __ldg(B.fwd_ptr + c) + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= __ldg(B.fwd_ptr + c + 1)) return;
  const int4 E = B.ent[e];
  factor_rows<TF, ONE_PASS, !ONE_PASS, DREG>(B.sys[E.x], E.y, E.z, E.w);
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
      factor_rows<TF, false>(B.sys[E.x], E.y, E.z, E.w);
    }
  }
}

}  // namespace opm
