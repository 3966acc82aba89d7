// sm_103a kernels of the BSR ILU0-BiCGStab path.
//
//  * k_spmv_*      blocked SpMV, y = A x (Section 4.3), one lane per block row
//                  on the warp-sliced layout, with the dot products the solver
//                  needs fused into its epilogue.
//  * k_factor      ILU0 decomposition (Algorithm 2) of the permuted matrix,
//                  fused with the value permutation (Algorithm 3's index copy).
//  * k_apply       ILU0 application (Algorithm 1): forward and backward block
//                  substitution in one launch, fused with the BiCGStab vector
//                  update that produces its right-hand side.
//  * k_update      x and r updates of BiCGStab plus the next reductions.
//
// The triangular kernels replace the paper's one launch per colour or level
// (Section 4.4) by one cooperative launch per preconditioner application:
// resident warps walk slices of 32 rows in schedule order, wait (bounded) on
// the ready flags of the other slices a slice reads, and publish their own.
// Dependencies inside one slice are resolved in rounds within the warp.
//
// Reductions are deterministic: every static-tiled kernel reduces its 256
// rows in a fixed butterfly, writes one partial per tile, and the last CTA to
// finish (atomic counter) sums the partials in index order and runs the
// scalar part of BiCGStab (alpha, omega, beta, the stopping rule).
#pragma once

#include <cstdint>

#include "opm_internal.h"

namespace opm {

enum SweepMode { kModePlain = 0, kModeP = 1, kModeS = 2 };

struct Sys {
  int32_t n, nslices;
  const int32_t *perm;
  const int32_t *a_rp, *a_col, *a_src;
  const int64_t *a_dst;
  double *a_val;
  const int32_t *l_rp, *l_col, *u_rp, *u_col;
  const int32_t *upd_ptr;
  const int64_t *upd_dst, *upd_src;
  void *lu;  // factor values (double or float): [L | U | Dinv slices]
  int64_t u_off, d_off;
  double *x, *r, *rh, *p, *v, *ph, *s, *sh, *t, *w;
  void *y;   // forward intermediate (factor precision)
  uint32_t *fflag, *bflag;
  const int32_t *fdep_ptr, *fdep, *bdep_ptr, *bdep;
  const uint32_t *fmask, *bmask;
  double *partials;
  DevState *st;
  uint64_t spin_limit_ns;
  int32_t skip_item;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_relaxed_i32(const int32_t *p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *flag == epoch.  Gives up (false) when another warp has
// reported an error, or sets OPM_ERR_TIMEOUT once limit_ns has passed.
__device__ __noinline__ bool wait_flag(const uint32_t *flag, uint32_t epoch, DevState *st,
                                       uint64_t limit_ns) {
  if (ld_acquire(flag) == epoch) return true;
  const uint64_t t0 = gtimer();
  unsigned nap = 32;
  for (uint32_t it = 1;; ++it) {
    __nanosleep(nap);  // back off so that waiting warps do not flood L2 with polls
    if (nap < 256) nap <<= 1;
    if (ld_acquire(flag) == epoch) return true;
    if ((it & 15u) == 0) {
      if (ld_relaxed_i32(&st->error) != 0) return false;
      if (gtimer() - t0 > limit_ns) {
        atomicCAS(&st->error, 0, (int32_t)OPM_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) {
  return __ldcg(p);
}

__device__ __forceinline__ bool running(const DevState *st) {
  return st->status == kRunning && st->error == 0;
}

// 3x3 inverse by the adjugate (the output is always written, non-finite for
// a singular block); returns false for a zero or non-finite determinant.
template <typename T>
__device__ __forceinline__ bool inv3(const T (&a)[9], T (&o)[9]) {
  T c0 = a[4] * a[8] - a[5] * a[7];
  T c1 = a[5] * a[6] - a[3] * a[8];
  T c2 = a[3] * a[7] - a[4] * a[6];
  T det = a[0] * c0 + a[1] * c1 + a[2] * c2;
  const bool ok = (det != T(0)) && isfinite(det);
  T id = T(1) / det;
  o[0] = c0 * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[3] = c1 * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[6] = c2 * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return ok;
}

// Deterministic reduction of NV values over a 256-thread CTA; the result is
// valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double *sm) {
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[w * NV + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double acc = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) acc += sm[ww * NV + q];
      v[q] = acc;
    }
  }
  __syncthreads();
}

// Per-tile partial, then the last CTA sums all partials in tile order.
// Returns true in the last CTA; tot is then valid in its thread 0.
template <int NV>
__device__ __forceinline__ bool last_cta_reduce(double (&v)[NV], double *partials, uint32_t *counter,
                                                double (&tot)[NV]) {
  __shared__ double sm[8 * NV];
  __shared__ int amlast;
  block_reduce<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[(size_t)blockIdx.x * NV + q] = v[q];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    amlast = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += __ldcg(partials + (size_t)b * NV + q);
  }
  block_reduce<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = acc[q];
    *counter = 0;
  }
  return true;
}

// y += A_row x for lane's row i of a warp-sliced part (FP64).  All lanes of
// the warp must call it; lanes with i >= n contribute nothing.
__device__ __forceinline__ void row_spmv(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                         const double *__restrict__ val, const double *__restrict__ x,
                                         int i, int n, double &y0, double &y1, double &y2) {
  const int lane = threadIdx.x & 31;
  const int s0 = i - lane;
  const int len = (i < n) ? rp[i + 1] - rp[i] : 0;
  int base = (s0 < n) ? rp[s0] : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  const unsigned lt = lanemask_lt();
  for (int k = 0; k < maxlen; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (len > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int j = __ldg(col + base + q);
      const double *a = val + 9ll * base + q;
      const double x0 = __ldg(x + 3ll * j), x1 = __ldg(x + 3ll * j + 1), x2 = __ldg(x + 3ll * j + 2);
      const double a0 = __ldg(a), a1 = __ldg(a + cnt), a2 = __ldg(a + 2 * cnt);
      const double a3 = __ldg(a + 3 * cnt), a4 = __ldg(a + 4 * cnt), a5 = __ldg(a + 5 * cnt);
      const double a6 = __ldg(a + 6 * cnt), a7 = __ldg(a + 7 * cnt), a8 = __ldg(a + 8 * cnt);
      y0 = fma(a0, x0, fma(a1, x1, fma(a2, x2, y0)));
      y1 = fma(a3, x0, fma(a4, x1, fma(a5, x2, y1)));
      y2 = fma(a6, x0, fma(a7, x1, fma(a8, x2, y2)));
    }
    base += __popc(m);
  }
}

// ------------------------------------------------------------ static kernels

// r = P b, r^ = r, x = p = v = 0, ||b||^2; the last CTA starts the solve.
__global__ void __launch_bounds__(256) k_setup(Sys S, const double *__restrict__ b_nat, double rtol,
                                               int32_t maxit) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  double acc[1] = {0.0};
  if (i < S.n) {
    const int o = S.perm[i];
    const double b0 = b_nat[3ll * o], b1 = b_nat[3ll * o + 1], b2 = b_nat[3ll * o + 2];
    double *r = S.r + 3ll * i, *rh = S.rh + 3ll * i;
    r[0] = b0; r[1] = b1; r[2] = b2;
    rh[0] = b0; rh[1] = b1; rh[2] = b2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S.x[3ll * i + c] = 0.0;
      S.p[3ll * i + c] = 0.0;
      S.v[3ll * i + c] = 0.0;
    }
    acc[0] = b0 * b0 + b1 * b1 + b2 * b2;
  }
  double tot[1];
  if (last_cta_reduce<1>(acc, S.partials, &S.st->red_count, tot) && threadIdx.x == 0) {
    DevState *st = S.st;
    const double n0 = sqrt(tot[0]);
    st->n0 = n0;
    st->tol = rtol * n0;
    st->maxit = maxit;
    st->k = 1;
    st->iters = 0;
    st->half = 0;
    st->error = 0;
    st->relres = 0.0;
    st->rho = tot[0];
    st->rho_prev = 1.0;
    st->alpha = 1.0;
    st->omega = 1.0;
    st->beta = tot[0];
    if (!isfinite(n0)) st->status = OPM_ERR_NONFINITE;
    else if (n0 == 0.0) st->status = OPM_OK;
    else if (maxit < 1) st->status = OPM_NOT_CONVERGED;
    else st->status = kRunning;
  }
}

// v = A p^ and (r^, v); alpha = rho / (r^, v).
__global__ void __launch_bounds__(256) k_spmv_v(Sys S) {
  if (!running(S.st)) return;
  const int i = blockIdx.x * 256 + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_spmv(S.a_rp, S.a_col, S.a_val, S.ph, i, S.n, y0, y1, y2);
  double acc[1] = {0.0};
  if (i < S.n) {
    double *v = S.v + 3ll * i;
    v[0] = y0; v[1] = y1; v[2] = y2;
    const double *rh = S.rh + 3ll * i;
    acc[0] = rh[0] * y0 + rh[1] * y1 + rh[2] * y2;
  }
  double tot[1];
  if (last_cta_reduce<1>(acc, S.partials, &S.st->red_count, tot) && threadIdx.x == 0) {
    DevState *st = S.st;
    st->rhv = tot[0];
    if (tot[0] == 0.0) {
      st->status = OPM_ERR_BREAKDOWN;
      st->iters = st->k;
    } else {
      st->alpha = st->rho / tot[0];
    }
  }
}

// t = A s^, (t,s), (t,t), (s,s); the half-step test and omega.
__global__ void __launch_bounds__(256) k_spmv_t(Sys S) {
  if (!running(S.st)) return;
  const int i = blockIdx.x * 256 + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_spmv(S.a_rp, S.a_col, S.a_val, S.sh, i, S.n, y0, y1, y2);
  double acc[3] = {0.0, 0.0, 0.0};
  if (i < S.n) {
    double *t = S.t + 3ll * i;
    t[0] = y0; t[1] = y1; t[2] = y2;
    const double *s = S.s + 3ll * i;
    acc[0] = y0 * s[0] + y1 * s[1] + y2 * s[2];
    acc[1] = y0 * y0 + y1 * y1 + y2 * y2;
    acc[2] = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  }
  double tot[3];
  if (last_cta_reduce<3>(acc, S.partials, &S.st->red_count, tot) && threadIdx.x == 0) {
    DevState *st = S.st;
    st->ts = tot[0];
    st->tt = tot[1];
    st->ss = tot[2];
    if (sqrt(tot[2]) <= st->tol) {
      st->half = 1;
    } else if (tot[1] == 0.0) {
      st->status = OPM_ERR_BREAKDOWN;
      st->iters = st->k;
    } else {
      const double om = tot[0] / tot[1];
      st->omega = om;
      if (om == 0.0) {
        st->status = OPM_ERR_BREAKDOWN;
        st->iters = st->k;
      }
    }
  }
}

// x += alpha p^ + omega s^, r = s - omega t, ||r||^2, (r^, r); stopping rule,
// then beta for the next iteration.
__global__ void __launch_bounds__(256) k_update(Sys S) {
  if (!running(S.st)) return;
  const int i = blockIdx.x * 256 + threadIdx.x;
  const DevState *cst = S.st;
  const double alpha = cst->alpha, omega = cst->omega;
  const int half = cst->half;
  double acc[2] = {0.0, 0.0};
  if (i < S.n) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t e = 3ll * i + c;
      if (half) {
        S.x[e] = fma(alpha, S.ph[e], S.x[e]);
      } else {
        S.x[e] = S.x[e] + fma(alpha, S.ph[e], omega * S.sh[e]);
        const double rr = fma(-omega, S.t[e], S.s[e]);
        S.r[e] = rr;
        acc[0] = fma(rr, rr, acc[0]);
        acc[1] = fma(S.rh[e], rr, acc[1]);
      }
    }
  }
  double tot[2];
  if (last_cta_reduce<2>(acc, S.partials, &S.st->red_count, tot) && threadIdx.x == 0) {
    DevState *st = S.st;
    const int k = st->k;
    if (half) {
      st->status = OPM_OK;
      st->iters = k;
      return;
    }
    st->rr = tot[0];
    st->rhr = tot[1];
    if (sqrt(tot[0]) <= st->tol) {
      st->status = OPM_OK;
      st->iters = k;
    } else if (k >= st->maxit) {
      st->status = OPM_NOT_CONVERGED;
      st->iters = k;
    } else if (tot[1] == 0.0) {
      st->status = OPM_ERR_BREAKDOWN;
      st->iters = k + 1;
    } else {
      st->rho_prev = st->rho;
      st->rho = tot[1];
      st->beta = (st->rho / st->rho_prev) * (st->alpha / st->omega);
      st->k = k + 1;
      st->iters = k;
    }
  }
}

// Final true residual ||b - A x|| / ||b|| in FP64 and x back to the caller's
// order.
__global__ void __launch_bounds__(256) k_finish(Sys S, const double *__restrict__ b_nat,
                                                double *__restrict__ x_nat) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_spmv(S.a_rp, S.a_col, S.a_val, S.x, i, S.n, y0, y1, y2);
  double acc[1] = {0.0};
  if (i < S.n) {
    const int o = S.perm[i];
    const double d0 = b_nat[3ll * o] - y0, d1 = b_nat[3ll * o + 1] - y1, d2 = b_nat[3ll * o + 2] - y2;
    acc[0] = d0 * d0 + d1 * d1 + d2 * d2;
#pragma unroll
    for (int c = 0; c < 3; ++c) x_nat[3ll * o + c] = S.x[3ll * i + c];
  }
  double tot[1];
  if (last_cta_reduce<1>(acc, S.partials, &S.st->red_count, tot) && threadIdx.x == 0) {
    DevState *st = S.st;
    st->relres = st->n0 > 0.0 ? sqrt(tot[0]) / st->n0 : 0.0;
  }
}

// y = A x in the caller's order (x already permuted into S.w).
__global__ void __launch_bounds__(256) k_spmv_plain(Sys S, const double *__restrict__ xp,
                                                    double *__restrict__ y_nat) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_spmv(S.a_rp, S.a_col, S.a_val, xp, i, S.n, y0, y1, y2);
  if (i < S.n) {
    const int o = S.perm[i];
    y_nat[3ll * o] = y0;
    y_nat[3ll * o + 1] = y1;
    y_nat[3ll * o + 2] = y2;
  }
}

// out[i] = in[perm[i]] (caller's order -> schedule order).
__global__ void __launch_bounds__(256) k_gather(Sys S, const double *__restrict__ in, double *__restrict__ out) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i < S.n) {
    const int o = S.perm[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3ll * i + c] = in[3ll * o + c];
  }
}

// out[perm[i]] = in[i] (schedule order -> caller's order).
__global__ void __launch_bounds__(256) k_scatter(Sys S, const double *__restrict__ in, double *__restrict__ out) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i < S.n) {
    const int o = S.perm[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3ll * o + c] = in[3ll * i + c];
  }
}

// ----------------------------------------------------- sync-free sweeps
//
// Sweep kernels are launched cooperatively with at most one wave of CTAs, so
// all their warps are resident at once.  Warp g of W handles slices g, g+W,
// g+2W, ... in increasing order (the backward sweep in decreasing order).  A
// slice only waits for slices that precede it in its sweep; those belong to
// resident warps that reach them without waiting on anything later, so every
// wait ends (and is bounded in time anyway).

struct Sweep {
  uint32_t epoch;
  uint64_t limit;
};

// Last CTA out advances the epoch for the next sweep launch.
__device__ __forceinline__ void sweep_exit(DevState *st, uint32_t epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->done, 1u) == gridDim.x - 1) {
      st->done = 0;
      st->epoch = epoch + 1;
      __threadfence();
    }
  }
}

__device__ __forceinline__ void signal(const Sys &S, uint32_t *flags, int s, int item, uint32_t epoch) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && item != S.skip_item) st_release(flags + s, epoch);
}

// Lanes poll the distinct slices listed for this slice, up to 32 at a time.
__device__ __forceinline__ void wait_slices(const Sys &S, const int32_t *__restrict__ ptr,
                                            const int32_t *__restrict__ list, const uint32_t *flags, int sl,
                                            const Sweep &sw) {
  const int lane = threadIdx.x & 31;
  const int d1 = ptr[sl + 1];
  for (int d = ptr[sl] + lane; d < d1; d += 32) wait_flag(flags + list[d], sw.epoch, S.st, sw.limit);
  __syncwarp();
}

template <typename TF>
struct Vec3 {
  TF c0, c1, c2;
};

template <typename TF>
__device__ __forceinline__ Vec3<TF> load3(const TF *p) {
  return {ldcg(p), ldcg(p + 1), ldcg(p + 2)};
}

// acc -= sum over the lane's row of a sliced part of B_ij v_j, v read from
// other warps' output (L2), two slabs per step for memory-level parallelism.
// Lanes with !act skip their loads; all lanes must call.
template <typename TF, typename TV>
__device__ __forceinline__ void row_sub(const int32_t *__restrict__ col, const TF *__restrict__ vals,
                                        const TV *vec, int len, int base0, int maxlen, bool act, TF &a0,
                                        TF &a1, TF &a2) {
  const unsigned lt = lanemask_lt();
  int base = base0;
  for (int k = 0; k < maxlen; k += 2) {
    const unsigned m0 = __ballot_sync(0xffffffffu, len > k);
    const unsigned m1 = __ballot_sync(0xffffffffu, len > k + 1);
    const int b0 = base, b1 = base + __popc(m0);
    base = b1 + __popc(m1);
    const bool u0 = act && len > k, u1 = act && len > k + 1;
    const int q0 = __popc(m0 & lt), q1 = __popc(m1 & lt);
    const int c0 = __popc(m0), c1 = __popc(m1);
    int j0 = 0, j1 = 0;
    if (u0) j0 = col[b0 + q0];
    if (u1) j1 = col[b1 + q1];
    if (u0) {
      const TF *B = vals + 9ll * b0 + q0;
      const TF v0 = (TF)ldcg(vec + 3ll * j0), v1 = (TF)ldcg(vec + 3ll * j0 + 1), v2 = (TF)ldcg(vec + 3ll * j0 + 2);
      a0 -= B[0] * v0 + B[c0] * v1 + B[2 * c0] * v2;
      a1 -= B[3 * c0] * v0 + B[4 * c0] * v1 + B[5 * c0] * v2;
      a2 -= B[6 * c0] * v0 + B[7 * c0] * v1 + B[8 * c0] * v2;
    }
    if (u1) {
      const TF *B = vals + 9ll * b1 + q1;
      const TF v0 = (TF)ldcg(vec + 3ll * j1), v1 = (TF)ldcg(vec + 3ll * j1 + 1), v2 = (TF)ldcg(vec + 3ll * j1 + 2);
      a0 -= B[0] * v0 + B[c1] * v1 + B[2 * c1] * v2;
      a1 -= B[3 * c1] * v0 + B[4 * c1] * v1 + B[5 * c1] * v2;
      a2 -= B[6 * c1] * v0 + B[7 * c1] * v1 + B[8 * c1] * v2;
    }
  }
}

// One slice of the forward substitution y_i = rhs_i - sum_{j<i} L_ij y_j,
// with the right-hand side formed on the fly (Algorithm 1, equation 3).
template <typename TF, int MODE>
__device__ __forceinline__ void fwd_slice(const Sys &S, int sl, const Sweep &sw, double alpha, double beta,
                                          double omega, const double *in) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const bool valid = i < n;
  TF *y = static_cast<TF *>(S.y);
  const TF *lu = static_cast<const TF *>(S.lu);
  double h0 = 0.0, h1 = 0.0, h2 = 0.0;
  unsigned dep = 0;
  int len = 0;
  if (valid) {
    const size_t e = 3ll * i;
    if (MODE == kModeP) {
      h0 = fma(beta, fma(-omega, S.v[e], S.p[e]), S.r[e]);
      h1 = fma(beta, fma(-omega, S.v[e + 1], S.p[e + 1]), S.r[e + 1]);
      h2 = fma(beta, fma(-omega, S.v[e + 2], S.p[e + 2]), S.r[e + 2]);
      S.p[e] = h0; S.p[e + 1] = h1; S.p[e + 2] = h2;
    } else if (MODE == kModeS) {
      h0 = fma(-alpha, S.v[e], S.r[e]);
      h1 = fma(-alpha, S.v[e + 1], S.r[e + 1]);
      h2 = fma(-alpha, S.v[e + 2], S.r[e + 2]);
      S.s[e] = h0; S.s[e + 1] = h1; S.s[e + 2] = h2;
    } else {
      h0 = in[e]; h1 = in[e + 1]; h2 = in[e + 2];
    }
    dep = S.fmask[i];
    len = S.l_rp[i + 1] - S.l_rp[i];
  }
  wait_slices(S, S.fdep_ptr, S.fdep, S.fflag, sl, sw);
  const int base0 = (s0 < n) ? S.l_rp[s0] : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  unsigned done = __ballot_sync(0xffffffffu, !valid);
  bool mine = !valid;
  while (done != 0xffffffffu) {
    const bool ready = !mine && ((dep & ~done) == 0);
    TF a0 = (TF)h0, a1 = (TF)h1, a2 = (TF)h2;
    row_sub<TF, TF>(S.l_col, lu, y, len, base0, maxlen, ready, a0, a1, a2);
    if (ready) {
      TF *yi = y + 3ll * i;
      yi[0] = a0; yi[1] = a1; yi[2] = a2;
      mine = true;
    }
    done |= __ballot_sync(0xffffffffu, ready);
    __syncwarp();
  }
  signal(S, S.fflag, sl, sl, sw.epoch);
}

// One slice of the backward substitution z_i = inv(U_ii)(y_i - sum_{j>i}
// U_ij z_j) (Algorithm 1, equation 4); z is written in FP64.
template <typename TF>
__device__ __forceinline__ void bwd_slice(const Sys &S, int sl, const Sweep &sw, double *z) {
  const int lane = threadIdx.x & 31;
  const int s0 = sl * 32;
  const int i = s0 + lane;
  const int n = S.n;
  const bool valid = i < n;
  const TF *y = static_cast<const TF *>(S.y);
  const TF *lu = static_cast<const TF *>(S.lu);
  unsigned dep = 0;
  int len = 0;
  if (valid) {
    dep = S.bmask[i];
    len = S.u_rp[i + 1] - S.u_rp[i];
  }
  if (lane == 0) wait_flag(S.fflag + sl, sw.epoch, S.st, sw.limit);
  wait_slices(S, S.bdep_ptr, S.bdep, S.bflag, sl, sw);
  Vec3<TF> yi = {TF(0), TF(0), TF(0)};
  if (valid) yi = load3(y + 3ll * i);
  const int base0 = (s0 < n) ? S.u_rp[s0] : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  const TF *D = lu + S.d_off + (int64_t)kSliceVals * sl + lane;
  TF d[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) d[c] = valid ? D[32 * c] : TF(0);
  unsigned done = __ballot_sync(0xffffffffu, !valid);
  bool mine = !valid;
  while (done != 0xffffffffu) {
    const bool ready = !mine && ((dep & ~done) == 0);
    TF a0 = yi.c0, a1 = yi.c1, a2 = yi.c2;
    row_sub<TF, double>(S.u_col, lu + S.u_off, z, len, base0, maxlen, ready, a0, a1, a2);
    if (ready) {
      double *zi = z + 3ll * i;
      zi[0] = (double)(d[0] * a0 + d[1] * a1 + d[2] * a2);
      zi[1] = (double)(d[3] * a0 + d[4] * a1 + d[5] * a2);
      zi[2] = (double)(d[6] * a0 + d[7] * a1 + d[8] * a2);
      mine = true;
    }
    done |= __ballot_sync(0xffffffffu, ready);
    __syncwarp();
  }
  signal(S, S.bflag, sl, S.nslices + (S.nslices - 1 - sl), sw.epoch);
}

// ILU0 application z = U^-1 L^-1 rhs in one cooperative launch: every warp
// runs its forward slices, then its backward slices.
template <typename TF, int MODE>
__global__ void __launch_bounds__(256) k_apply(Sys S, const double *in, double *out) {
  DevState *st = S.st;
  const uint32_t epoch = st->epoch;
  const bool run = (MODE == kModePlain) || running(st);
  if (run) {
    const Sweep sw{epoch, S.spin_limit_ns};
    const double alpha = st->alpha, beta = st->beta, omega = st->omega;
    double *z = (MODE == kModeP) ? S.ph : (MODE == kModeS) ? S.sh : out;
    const int ns = S.nslices;
    const int W = gridDim.x * (blockDim.x >> 5);
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int sl = g; sl < ns; sl += W) fwd_slice<TF, MODE>(S, sl, sw, alpha, beta, omega, in);
    for (int q = g; q < ns; q += W) bwd_slice<TF>(S, ns - 1 - q, sw, z);
  }
  sweep_exit(st, epoch);
}

// ILU0 decomposition (Algorithm 2) of the permuted matrix, one slice per
// warp step in schedule order, fused with the value permutation: with
// vals_user, block w of the permuted matrix is copied from the caller's
// block a_src[w] (Algorithm 3's index copy) into both A and the factors.
template <typename TF>
__global__ void __launch_bounds__(256) k_factor(Sys S, const double *__restrict__ vals_user) {
  DevState *st = S.st;
  const uint32_t epoch = st->epoch;
  const Sweep sw{epoch, S.spin_limit_ns};
  const int n = S.n;
  TF *lu = static_cast<TF *>(S.lu);
  const unsigned lt = lanemask_lt();
  const int lane = threadIdx.x & 31;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int sl = g; sl < S.nslices; sl += W) {
    const int s0 = sl * 32;
    const int i = s0 + lane;
    const bool valid = i < n;
    // ---- copy phase: A's row into A (sliced) and into L / D / U slots
    {
      const int len = valid ? S.a_rp[i + 1] - S.a_rp[i] : 0;
      int base = (s0 < n) ? S.a_rp[s0] : 0;
      const int maxlen = __reduce_max_sync(0xffffffffu, len);
      for (int k = 0; k < maxlen; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, len > k);
        if (len > k) {
          const int cnt = __popc(m);
          const int q = __popc(m & lt);
          const int w = base + q;
          const int64_t dst = S.a_dst[w];
          const int64_t doff = dst >> 6;
          const int dstr = (int)(dst & 63);
          double *av = S.a_val + 9ll * base + q;
          double e[9];
          if (vals_user) {
            const double *src = vals_user + 9ll * S.a_src[w];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
              e[c] = __ldg(src + c);
              av[c * cnt] = e[c];
            }
          } else {
#pragma unroll
            for (int c = 0; c < 9; ++c) e[c] = av[c * cnt];
          }
#pragma unroll
          for (int c = 0; c < 9; ++c) lu[doff + (int64_t)c * dstr] = (TF)e[c];
        }
        base += __popc(m);
      }
    }
    // ---- dependencies on earlier rows (the pivots k < i of row i)
    const unsigned dep = valid ? S.fmask[i] : 0u;
    wait_slices(S, S.fdep_ptr, S.fdep, S.fflag, sl, sw);
    const int len = valid ? S.l_rp[i + 1] - S.l_rp[i] : 0;
    const int lrow = valid ? S.l_rp[i] : 0;
    const int base0 = (s0 < n) ? S.l_rp[s0] : 0;
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    unsigned done = __ballot_sync(0xffffffffu, !valid);
    bool mine = !valid;
    while (done != 0xffffffffu) {
      const bool ready = !mine && ((dep & ~done) == 0);
      int base = base0;
      for (int k = 0; k < maxlen; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, len > k);
        if (ready && len > k) {
          const int cnt = __popc(m);
          const int q = __popc(m & lt);
          const int kc = S.l_col[base + q];
          TF *Lp = lu + 9ll * base + q;
          const TF *Dk = lu + S.d_off + (int64_t)kSliceVals * (kc >> 5) + (kc & 31);
          TF a[9], d[9], l[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            a[c] = Lp[c * cnt];
            d[c] = ldcg(Dk + 32 * c);
          }
          // L_ik = A_ik * inv(U_kk)
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              l[3 * r + c] = a[3 * r] * d[c] + a[3 * r + 1] * d[3 + c] + a[3 * r + 2] * d[6 + c];
#pragma unroll
          for (int c = 0; c < 9; ++c) Lp[c * cnt] = l[c];
          // A_ij -= L_ik * U_kj for the listed j
          const int u1 = S.upd_ptr[lrow + k + 1];
          for (int u = S.upd_ptr[lrow + k]; u < u1; ++u) {
            const int64_t ds = S.upd_dst[u], ss = S.upd_src[u];
            TF *Ap = lu + (ds >> 6);
            const int dstr = (int)(ds & 63);
            const TF *Up = lu + (ss >> 6);
            const int sstr = (int)(ss & 63);
            TF uu[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) uu[c] = ldcg(Up + c * sstr);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
              for (int c = 0; c < 3; ++c)
                Ap[(3 * r + c) * dstr] -=
                    l[3 * r] * uu[c] + l[3 * r + 1] * uu[3 + c] + l[3 * r + 2] * uu[6 + c];
          }
        }
        base += __popc(m);
      }
      if (ready) {
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
        mine = true;
      }
      done |= __ballot_sync(0xffffffffu, ready);
      __syncwarp();
    }
    signal(S, S.fflag, sl, sl, epoch);
  }
  sweep_exit(st, epoch);
}

}  // namespace opm
