// sm_103a kernels of the BSR ILU0-BiCGStab path: the shared device data,
// helpers and reductions, and the row-parallel kernels.
//
//  * k_spmv_*        blocked SpMV, y = A x (Section 4.3), one lane per block
//                    row on the warp-sliced layout, with the dot products the
//                    solver needs fused into the epilogue.
//  * k_update        x and r updates of BiCGStab and the next reductions.
//  * k_setup, k_finish, control kernels.
//
// The ILU0 decomposition (Algorithm 2, k_factor*) is in factor.cuh, the ILU0
// application (Algorithm 1, k_fwd/bwd_phase, k_apply) in sweeps.cuh.
//
// Every kernel works on a batch of independent systems described in device
// memory (a single solve is a batch of one).  Work is split per system into
// fixed units -- 32-row slices for the sweeps, 256- or 1024-row tiles for the
// row-parallel kernels -- so a system's arithmetic, including the order of
// every reduction, is the same alone and inside any batch.
//
// Phases: the schedule's row order is cut into maximal runs of rows none of
// which reads another row of its run (the levels or the colours, Section
// 4.4).  The sweeps walk the phases in order, either one launch per phase
// or one cooperative launch with a bounded grid barrier between phases.
//
// Reductions: per system in a fixed order (see red_end and
// last_cta_reduce); the warp or CTA that completes a system's sum runs the
// scalar part of BiCGStab (alpha, omega, beta, the stopping rule).
#pragma once

#include <cstdint>

#include "opm_internal.h"

namespace opm {

enum SweepMode { kModePlain = 0, kModeP = 1, kModeS = 2 };

// One system's device data.  The last group of fields is set per call.
struct Sys {
  int32_t n, nslices, ntiles, nphases;
  int32_t ntiles_s;  // 256-row tiles of the SpMV kernels
  int32_t pad0;
  const int32_t *perm;
  const int32_t *a_rp, *a_col, *a_src;
  const int64_t *a_dst;
  double *a_val;
  const int32_t *l_rp, *l_col, *u_rp, *u_col;
  const int32_t *upd_ptr;
  const int64_t *upd_dst, *upd_src;
  const uint2 *sl_mask;  // per slice: (rows without U blocks, rows whose y is read later)
  const uint32_t *fz_mask;  // per slice: rows the factorisation walks in one pass
  const int64_t *a_aux;     // per A block: slot of U_ki for a one-pass row's L block (i,k), else -1
  // products after an application (Analysis::sp_mask, sp_len): per slice
  // (rows with (A p^)_i = p_i, rows taking their upper sum from the
  // backward sweep); per row the leading blocks of A the product walks
  const uint2 *sp_mask;
  const int32_t *sp_len;
  // per row: sum_{j>i} U_ij z_j of the last BiCGStab application, stored by
  // the backward sweep for the rows of sp_mask.y.  NULL: the products walk
  // all of A (FP32 factors, Jacobi triangular sweeps, or turned off)
  double *uz;
  // standard wells applied separately (nwells = 0: none)
  int32_t nwells, pad1;
  const int32_t *w_ptr;     // [nwells+1] perforations of each well
  const int32_t *w_cell;    // [nperf] perforated cell (schedule order)
  const int32_t *w_of;      // [nperf] well of each perforation
  const double *w_B, *w_C;  // [nperf][12] 4x3 row-major
  const double *w_Dinv;     // [nwells][16] 4x4 row-major
  const int32_t *w_rptr;    // [n+1] perforations of each row (into w_rperf)
  const int32_t *w_rperf;   // perforation indices by row
  const uint32_t *w_mask;   // per slice: rows with perforations
  double *w_t2;             // [nwells][4] inv(D) B x of the current product
  const int32_t *w_rows;    // [nwrows] perforated rows, ascending
  int32_t nwrows, pad2;
  double *w_corr;           // [3n] sum of C_p^T t2 over row i's perforations (perforated rows only)
  void *lu;  // factor values (double or float): [L | U | Dinv slices]
  void *lu2; // second factor buffer of the iterative ILU0 (cp_sweeps > 0), else NULL
  int64_t u_off, d_off;
  double *x, *r, *rh, *p, *v, *ph, *s, *sh, *t, *w;
  void *y;   // forward intermediate (factor precision)
  void *y2;  // Jacobi triangular sweeps (tri_sweeps > 0): second forward iterate, else NULL
  double *z2;  // Jacobi triangular sweeps: second backward iterate, else NULL
  double *partials;      // per tile: up to 4 partial sums
  double *grp_partials;  // per group of 32 tiles: up to 4 partial sums
  uint32_t *grp_count;   // per group of 32 tiles: tiles done (0 between kernels)
  DevState *st;
  // per call
  const double *b_in;    // right-hand side, or the input of spmv / ilu_apply (caller's order)
  double *x_out;         // solution, or the output of spmv / ilu_apply (caller's order)
  const double *vals_in; // new matrix values for the factorisation (NULL: refactor A)
  double rtol;
  int32_t maxit;
  int32_t skip;          // the system sits this batch launch out: no kernel touches it
};

// A launchable set of systems (kernel parameter).
struct Batch {
  const Sys *sys;         // [nsys]
  const int4 *ent;        // sweep work: (system, slice, first row, last row + 1)
  const int32_t *fwd_ptr; // [nphases + 1]: forward entries of phase c
  const int32_t *bwd_ptr; // [nphases + 1]: backward entries of phase c
  const int2 *tiles;      // (system, 1024-row tile) for the streaming kernels
  const int2 *tiles_s;    // (system, 256-row tile) for the SpMV kernels
  const int4 *all_ent;    // every slice of every system: (system, slice, 0, n)
  int32_t nall, pad;
  uint32_t *bar;          // grid barrier: arrivals at bar[0], generation at bar[32]
  int32_t nsys, nphases, ntiles, ntiles_s;
  int32_t skip_cta;       // test hook: this CTA never arrives at grid barriers (-1: off)
  uint64_t spin_limit_ns;
};

// Per-system outcome gathered for the host.
struct Result {
  int32_t status, iters, err_row, pad;
  double relres;
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

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch.  pdl_trigger lets the next kernel of the
// stream begin launching at once, so its CTAs become resident while this
// one runs; pdl_wait blocks until the preceding kernel has completed and its
// writes are visible.  A kernel reads nothing written by earlier kernels of
// the solve before its pdl_wait (only data that is constant for the whole
// solve: factors, index arrays, descriptors).  Both are no-ops for a kernel
// launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_trigger();
  pdl_wait();
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

// ------------------------------------------------------------ reductions
//
// A per-system sum of NV values without CTA-wide barriers, in a fixed order:
// every warp sums its lanes (xor butterfly); the last warp of the CTA to
// finish adds the CTA's warp sums in warp order (the tile's partial); the
// last tile of each group of 32 tiles adds the group's tile partials (xor
// butterfly over 32 lanes); the last group of the system adds the group
// partials (strided over the lanes, then the butterfly).  Warps that are not
// last simply exit, so no warp idles at a barrier, and the system's final
// sum is one warp's work.  The order depends only on the tile index, so a
// system's sums are the same alone and inside any batch.

constexpr int kMaxWarps = 8;  // warps per CTA of the reducing kernels (256 threads)

template <int NV>
struct RedShared {
  double wsum[kMaxWarps][NV];
  unsigned count;
};

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
}

// Called by every thread at kernel start (one CTA barrier).
template <int NV>
__device__ __forceinline__ void red_begin(RedShared<NV> &rs) {
  if (threadIdx.x == 0) rs.count = 0;
  __syncthreads();
}

// The CTA's last warp: tile partial, group partial, system sum (kept out of
// line: it runs once per CTA, and inlined it raises the register count of
// the whole kernel).
template <int NV>
__device__ __noinline__ bool red_tail(RedShared<NV> &rs, const Sys &S, int tile, int ntiles, int nw, int lane,
                                      double (&tot)[NV]) {
  unsigned t = 0;
  // the tile's partial, warps in order
  const int g = tile >> 5, ng = (ntiles + 31) >> 5, gsize = min(32, ntiles - 32 * g);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double p = 0.0;
#pragma unroll 1
      for (int ww = 0; ww < nw; ++ww) p += rs.wsum[ww][q];
      S.partials[(size_t)tile * NV + q] = p;
    }
    __threadfence();
    t = atomicAdd(&S.grp_count[g], 1u);
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != (unsigned)gsize - 1) return false;
  __threadfence();
  // the group's partial: lane l holds tile 32 g + l
  double gp[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) gp[q] = lane < gsize ? __ldcg(S.partials + (size_t)(32 * g + lane) * NV + q) : 0.0;
  warp_sum<NV>(gp);
  if (lane == 0) {
    S.grp_count[g] = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) S.grp_partials[(size_t)g * NV + q] = gp[q];
    __threadfence();
    t = atomicAdd(&S.st->red_count, 1u);
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != (unsigned)ng - 1) return false;
  __threadfence();
  // the system's sum: groups strided over the lanes, then the butterfly
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = 0.0;
#pragma unroll 1
  for (int gg = lane; gg < ng; gg += 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] += __ldcg(S.grp_partials + (size_t)gg * NV + q);
  }
  warp_sum<NV>(tot);
  if (lane == 0) S.st->red_count = 0;
  return true;
}

// Adds the calling warp's values v to tile `tile` of a system with ntiles
// tiles.  Returns true in every lane of the one warp that completes the
// system's sum; tot is then valid in all its lanes.
template <int NV>
__device__ __forceinline__ bool red_end(double (&v)[NV], RedShared<NV> &rs, const Sys &S, int tile, int ntiles,
                                        double (&tot)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  warp_sum<NV>(v);
  unsigned t = 0;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) rs.wsum[w][q] = v[q];
    __threadfence_block();
    t = atomicAdd(&rs.count, 1u);
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != (unsigned)nw - 1) return false;
  __threadfence_block();
  return red_tail<NV>(rs, S, tile, ntiles, nw, lane, tot);
}

// The second form: a CTA-wide tree in shared memory (values leave the
// registers at once), then the system's last CTA sums the tile partials in
// tile order.  k_spmv_t's three sums use it: measured on GB300 its launch
// takes 147 us this way against 172 us with red_end (same arithmetic order
// class, both deterministic), while the one- and two-value kernels are
// faster with red_end (k_spmv_v 135 against 140 us).
constexpr int kRedThreads = 256;

template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double *sm) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sm[q * kRedThreads + t] = v[q];
  __syncthreads();
#pragma unroll
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int q = 0; q < NV; ++q) sm[q * kRedThreads + t] += sm[q * kRedThreads + t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sm[q * kRedThreads];
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ bool last_cta_reduce(double (&v)[NV], const Sys &S, int tile, int ntiles,
                                                double (&tot)[NV]) {
  __shared__ double sm[kRedThreads * NV];
  __shared__ int amlast;
  block_reduce<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) S.partials[(size_t)tile * NV + q] = v[q];
    __threadfence();
    const unsigned t = atomicAdd(&S.st->red_count, 1u);
    amlast = (t == (unsigned)ntiles - 1);
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
#pragma unroll 8
  for (int b = threadIdx.x; b < ntiles; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += __ldcg(S.partials + (size_t)b * NV + q);
  }
  block_reduce<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = acc[q];
    S.st->red_count = 0;
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
      // the matrix is read once per product: streaming loads leave L2 to the vectors
      const int j = __ldcs(col + base + q);
      const double *a = val + 9ll * base + q;
      const double x0 = __ldg(x + 3ll * j), x1 = __ldg(x + 3ll * j + 1), x2 = __ldg(x + 3ll * j + 2);
      const double a0 = __ldcs(a), a1 = __ldcs(a + cnt), a2 = __ldcs(a + 2 * cnt);
      const double a3 = __ldcs(a + 3 * cnt), a4 = __ldcs(a + 4 * cnt), a5 = __ldcs(a + 5 * cnt);
      const double a6 = __ldcs(a + 6 * cnt), a7 = __ldcs(a + 7 * cnt), a8 = __ldcs(a + 8 * cnt);
      y0 = fma(a0, x0, fma(a1, x1, fma(a2, x2, y0)));
      y1 = fma(a3, x0, fma(a4, x1, fma(a5, x2, y1)));
      y2 = fma(a6, x0, fma(a7, x1, fma(a8, x2, y2)));
    }
    base += __popc(m);
  }
}

// Standard wells kept separate (Section 4.6): y -= C^T inv(D) B x.  k_wells
// runs before each product, one CTA per system: first t2_w = inv(D_w)
// (B_w x) for every well (one warp per well, lanes over the perforations,
// fixed butterfly order), then, for every perforated row, corr_i = the sum
// of C_p^T t2_w over its perforations (in perforation order).  The SpMV
// kernels start a perforated row's sum at -corr_i.

// The vector a product reads: 0 p^, 1 s^, 2 x, 3 w (caller's input), 4 t.
__device__ __forceinline__ const double *operator_input(const Sys &S, int which) {
  return which == 0 ? S.ph : which == 1 ? S.sh : which == 2 ? S.x : which == 3 ? S.w : S.t;
}

__global__ void __launch_bounds__(256) k_wells(Batch B, int which) {
  pdl_enter();
  const Sys &S = B.sys[blockIdx.x];
  const int nw = S.nwells;
  if (nw == 0 || S.skip) return;
  const double *x = operator_input(S, which);
  const int lane = threadIdx.x & 31;
  for (int w = threadIdx.x >> 5; w < nw; w += blockDim.x >> 5) {
    double t1[4] = {0.0, 0.0, 0.0, 0.0};
    const int p1 = __ldg(S.w_ptr + w + 1);
    for (int p = __ldg(S.w_ptr + w) + lane; p < p1; p += 32) {
      const int c = __ldg(S.w_cell + p);
      const double *Bp = S.w_B + 12ll * p;
      const double x0 = __ldcg(x + 3ll * c), x1 = __ldcg(x + 3ll * c + 1), x2 = __ldcg(x + 3ll * c + 2);
#pragma unroll
      for (int r = 0; r < 4; ++r)
        t1[r] = fma(__ldg(Bp + 3 * r), x0, fma(__ldg(Bp + 3 * r + 1), x1, fma(__ldg(Bp + 3 * r + 2), x2, t1[r])));
    }
    warp_sum<4>(t1);
    if (lane < 4) {
      const double *Dw = S.w_Dinv + 16ll * w + 4 * lane;
      S.w_t2[4ll * w + lane] =
          fma(__ldg(Dw), t1[0], fma(__ldg(Dw + 1), t1[1], fma(__ldg(Dw + 2), t1[2], __ldg(Dw + 3) * t1[3])));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < S.nwrows; k += blockDim.x) {
    const int i = __ldg(S.w_rows + k);
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    for (int q = __ldg(S.w_rptr + i); q < __ldg(S.w_rptr + i + 1); ++q) {
      const int p = __ldg(S.w_rperf + q);
      const double *t2 = S.w_t2 + 4ll * __ldg(S.w_of + p);
      const double *Cp = S.w_C + 12ll * p;
      const double a = t2[0], b = t2[1], c = t2[2], d = t2[3];
      c0 += fma(__ldg(Cp), a, fma(__ldg(Cp + 3), b, fma(__ldg(Cp + 6), c, __ldg(Cp + 9) * d)));
      c1 += fma(__ldg(Cp + 1), a, fma(__ldg(Cp + 4), b, fma(__ldg(Cp + 7), c, __ldg(Cp + 10) * d)));
      c2 += fma(__ldg(Cp + 2), a, fma(__ldg(Cp + 5), b, fma(__ldg(Cp + 8), c, __ldg(Cp + 11) * d)));
    }
    S.w_corr[3ll * i] = c0;
    S.w_corr[3ll * i + 1] = c1;
    S.w_corr[3ll * i + 2] = c2;
  }
}

// The system operator's row: y = (A x)_i minus the wells' corr_i when row i
// is perforated (the sum starts at -corr_i).
__device__ __forceinline__ void row_operator(const Sys &S, const double *__restrict__ x, int i, double &y0,
                                             double &y1, double &y2) {
  if (S.nwells > 0 && i < S.n && ((__ldg(S.w_mask + (i >> 5)) >> (i & 31)) & 1u)) {
    y0 = -__ldcg(S.w_corr + 3ll * i);
    y1 = -__ldcg(S.w_corr + 3ll * i + 1);
    y2 = -__ldcg(S.w_corr + 3ll * i + 2);
  }
  row_spmv(S.a_rp, S.a_col, S.a_val, x, i, S.n, y0, y1, y2);
}

// y += the first lead blocks of lane's row i of A's warp-sliced layout
// (FP64).  The slab layout is walked with every row's full length; lanes
// issue loads only for their first lead blocks, and the walk stops after
// the longest lead of the warp.  All lanes of the warp must call it.
__device__ __forceinline__ void row_spmv_lead(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                              const double *__restrict__ val, const double *__restrict__ x,
                                              int i, int n, int lead, double &y0, double &y1, double &y2) {
  const int maxlead = __reduce_max_sync(0xffffffffu, lead);
  if (maxlead == 0) return;  // warp-uniform: no lane walks a block
  const int lane = threadIdx.x & 31;
  const int s0 = i - lane;
  const int len = (i < n) ? rp[i + 1] - rp[i] : 0;
  int base = (s0 < n) ? rp[s0] : 0;
  const unsigned lt = lanemask_lt();
  for (int k = 0; k < maxlead; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, len > k);
    if (lead > k) {
      const int cnt = __popc(m);
      const int q = __popc(m & lt);
      const int j = __ldcs(col + base + q);
      const double *a = val + 9ll * base + q;
      const double x0 = __ldg(x + 3ll * j), x1 = __ldg(x + 3ll * j + 1), x2 = __ldg(x + 3ll * j + 2);
      const double a0 = __ldcs(a), a1 = __ldcs(a + cnt), a2 = __ldcs(a + 2 * cnt);
      const double a3 = __ldcs(a + 3 * cnt), a4 = __ldcs(a + 4 * cnt), a5 = __ldcs(a + 5 * cnt);
      const double a6 = __ldcs(a + 6 * cnt), a7 = __ldcs(a + 7 * cnt), a8 = __ldcs(a + 8 * cnt);
      y0 = fma(a0, x0, fma(a1, x1, fma(a2, x2, y0)));
      y1 = fma(a3, x0, fma(a4, x1, fma(a5, x2, y1)));
      y2 = fma(a6, x0, fma(a7, x1, fma(a8, x2, y2)));
    }
    base += __popc(m);
  }
}

// The operator's row right after a BiCGStab application xh = inv(LU) xin
// (REUSE; without it, row_operator).  ILU0 gives (LU)_ij = A_ij on the
// pattern.  A row with no block left of its diagonal and all blocks in the
// preconditioner has an empty L row and U's row equal to A's, so
// (A xh)_i = (U xh)_i = (L U xh)_i = xin_i: no product at all.  A row whose
// upper blocks all equal U's (sp_mask.y) starts from the backward sweep's
// sum_{j>i} U_ij xh_j (uz) and adds its diagonal and lower blocks.  Equal
// to row_operator in exact arithmetic; the wells' term is applied as there.
template <bool REUSE>
__device__ __forceinline__ void row_operator_applied(const Sys &S, const double *__restrict__ xh,
                                                     const double *__restrict__ xin, int i, double &y0,
                                                     double &y1, double &y2) {
  if (!REUSE) {
    row_operator(S, xh, i, y0, y1, y2);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int n = S.n;
  int lead = 0;
  if (i < n) {
    if (S.nwells > 0 && ((__ldg(S.w_mask + (i >> 5)) >> lane) & 1u)) {
      y0 = -__ldcg(S.w_corr + 3ll * i);
      y1 = -__ldcg(S.w_corr + 3ll * i + 1);
      y2 = -__ldcg(S.w_corr + 3ll * i + 2);
    }
    const uint2 M = __ldg(S.sp_mask + (i >> 5));
    lead = __ldg(S.sp_len + i);
    const double *e = ((M.x >> lane) & 1u) ? xin + 3ll * i : ((M.y >> lane) & 1u) ? S.uz + 3ll * i : nullptr;
    if (e) {
      y0 += __ldcg(e);
      y1 += __ldcg(e + 1);
      y2 += __ldcg(e + 2);
    }
  }
  row_spmv_lead(S.a_rp, S.a_col, S.a_val, xh, i, n, lead, y0, y1, y2);
}

// ------------------------------------------------------------ tile kernels
//
// One CTA per (system, tile).  Streaming kernels use tiles of kTileRows =
// 1024 rows and 256 threads in 4 passes (thread t: rows t, t + 256, t + 512,
// t + 768 of the tile); SpMV kernels use tiles of kSpmvRows = 256 rows, one
// row per thread, so that their last partial wave stays short.

#define OPM_TILE(B, S, lt)                  \
  const int2 tile_ = (B).tiles[blockIdx.x]; \
  const Sys &S = (B).sys[tile_.x];          \
  const int lt = tile_.y

#define OPM_TILE_S(B, S, lt)                  \
  const int2 tile_ = (B).tiles_s[blockIdx.x]; \
  const Sys &S = (B).sys[tile_.x];            \
  const int lt = tile_.y

#define OPM_TILE_ROWS(i, lt) \
  for (int pass_ = 0, i = (lt) * kTileRows + threadIdx.x; pass_ < 4; ++pass_, i += 256)

// Starts a solve: r = P b, r^ = r, x = p = v = 0, ||b||^2; the system's
// last CTA sets the scalars.  A factorisation error makes the solve fail.
// The solve state from ||b||^2 (bb) and the factorisation's outcome.
__device__ __forceinline__ void setup_scalars(const Sys &S, DevState *st, double bb) {
  const double n0 = sqrt(bb);
  st->n0 = n0;
  st->tol = S.rtol * n0;
  st->maxit = S.maxit;
  st->k = 1;
  st->iters = 0;
  st->half = 0;
  st->error = 0;
  st->relres = 0.0;
  st->rho = bb;
  st->rho_prev = 1.0;
  st->alpha = 1.0;
  st->omega = 1.0;
  st->beta = bb;
  if (st->ferror != 0) st->status = st->ferror;
  else if (!isfinite(n0)) st->status = OPM_ERR_NONFINITE;
  else if (n0 == 0.0) st->status = OPM_OK;
  else if (S.maxit < 1) st->status = OPM_NOT_CONVERGED;
  else st->status = kRunning;
}

// FINAL: the last CTA also sets the solve state.  Without FINAL (beside a
// running factorisation) it only records ||b||^2 and leaves the state and
// the grid barrier to k_start.
template <bool FINAL>
__global__ void __launch_bounds__(256, 6) k_setup(Batch B) {
  __shared__ RedShared<1> rs_;
  red_begin<1>(rs_);
  OPM_TILE(B, S, lt);
  if (FINAL && blockIdx.x == 0 && threadIdx.x == 0) B.bar[0] = 0;
  if (S.skip) return;
  double acc[1] = {0.0};
  const double *__restrict__ b_in = S.b_in;
  const int32_t *__restrict__ perm = S.perm;
  double *__restrict__ r = S.r, *__restrict__ rh = S.rh, *__restrict__ x = S.x, *__restrict__ p = S.p,
                       *__restrict__ v = S.v;
  const int n = S.n;
  OPM_TILE_ROWS(i, lt) {
    if (i < n) {
      const int o = __ldg(perm + i);
      const double b0 = __ldg(b_in + 3ll * o), b1 = __ldg(b_in + 3ll * o + 1), b2 = __ldg(b_in + 3ll * o + 2);
      const size_t e0 = 3ll * i;
      r[e0] = b0; r[e0 + 1] = b1; r[e0 + 2] = b2;
      rh[e0] = b0; rh[e0 + 1] = b1; rh[e0 + 2] = b2;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x[e0 + c] = 0.0;
        p[e0 + c] = 0.0;
        v[e0 + c] = 0.0;
      }
      acc[0] = fma(b0, b0, fma(b1, b1, fma(b2, b2, acc[0])));
    }
  }
  double tot[1];
  if (red_end<1>(acc, rs_, S, lt, S.ntiles, tot) && (threadIdx.x & 31) == 0) {
    if (FINAL) setup_scalars(S, S.st, tot[0]);
    else S.st->bb = tot[0];
  }
}

// Joins the factorisation and k_setup<false>: the solve state of every
// system, then the grid barrier's reset.
__global__ void k_start(Batch B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) B.bar[0] = 0;
  if (s < B.nsys && !B.sys[s].skip) setup_scalars(B.sys[s], B.sys[s].st, B.sys[s].st->bb);
}

// v = A p^ and (r^, v); alpha = rho / (r^, v).  REUSE: the product takes
// the application's sums where the factors allow (row_operator_applied).
template <bool REUSE>
__global__ void __launch_bounds__(256, 8) k_spmv_v(Batch B) {
  __shared__ RedShared<1> rs_;
  red_begin<1>(rs_);
  pdl_enter();
  OPM_TILE_S(B, S, lt);
  if (!running(S.st)) return;
  double acc[1] = {0.0};
  const int i = lt * kSpmvRows + threadIdx.x;
  {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    row_operator_applied<REUSE>(S, S.ph, S.p, i, y0, y1, y2);
    if (i < S.n) {
      double *v = S.v + 3ll * i;
      v[0] = y0; v[1] = y1; v[2] = y2;
      const double *rh = S.rh + 3ll * i;
      acc[0] = fma(rh[0], y0, fma(rh[1], y1, fma(rh[2], y2, acc[0])));
    }
  }
  double tot[1];
  if (red_end<1>(acc, rs_, S, lt, S.ntiles_s, tot) && (threadIdx.x & 31) == 0) {
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

// t = A s^, (t,s), (t,t), (s,s); the half-step test and omega.  REUSE as
// for k_spmv_v.  WIDE: eight CTAs per SM (32 registers; with REUSE its
// three sums spill 56 bytes per thread), for launches with more tiles than
// six CTAs per SM hold; otherwise (REUSE) six CTAs per SM and no spill,
// which a small system's latency-bound product prefers.
template <bool REUSE, bool WIDE = true>
__global__ void __launch_bounds__(256, (REUSE && !WIDE) ? 6 : 8) k_spmv_t(Batch B) {

  pdl_enter();
  OPM_TILE_S(B, S, lt);
  if (!running(S.st)) return;
  double acc[3] = {0.0, 0.0, 0.0};
  const int i = lt * kSpmvRows + threadIdx.x;
  {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    row_operator_applied<REUSE>(S, S.sh, S.s, i, y0, y1, y2);
    if (i < S.n) {
      double *t = S.t + 3ll * i;
      t[0] = y0; t[1] = y1; t[2] = y2;
      const double *s = S.s + 3ll * i;
      const double s0 = s[0], s1 = s[1], s2 = s[2];
      acc[0] = fma(y0, s0, fma(y1, s1, fma(y2, s2, acc[0])));
      acc[1] = fma(y0, y0, fma(y1, y1, fma(y2, y2, acc[1])));
      acc[2] = fma(s0, s0, fma(s1, s1, fma(s2, s2, acc[2])));
    }
  }
  double tot[3];
  if (last_cta_reduce<3>(acc, S, lt, S.ntiles_s, tot) && threadIdx.x == 0) {
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
// then beta for the next iteration.  A row's 18 loads issue before its
// stores (the vectors are distinct buffers), at four CTAs per SM (64
// registers).  Measured at the 949,871-cell system (A/B on one box, event
// timed): 54.8 us with one entry's loads at a time at eight CTAs per SM,
// 51.4 us this way; 57.6 at six CTAs per SM, 62.7 at three, 60.0 with two
// rows' loads at once at two.
__global__ void __launch_bounds__(256, 4) k_update(Batch B) {
  __shared__ RedShared<2> rs_;
  red_begin<2>(rs_);
  pdl_enter();
  OPM_TILE(B, S, lt);
  if (!running(S.st)) return;
  const DevState *cst = S.st;
  const double alpha = cst->alpha, omega = cst->omega;
  const int half = cst->half;
  double acc[2] = {0.0, 0.0};
  // the eight vectors are distinct buffers: a row's 18 loads issue before
  // any of its stores
  double *__restrict__ xv = S.x;
  double *__restrict__ rv = S.r;
  const double *__restrict__ phv = S.ph;
  const double *__restrict__ shv = S.sh;
  const double *__restrict__ tv = S.t;
  const double *__restrict__ sv = S.s;
  const double *__restrict__ rhv = S.rh;
  OPM_TILE_ROWS(i, lt) {
    if (i < S.n) {
      const size_t e = 3ll * i;
      if (half) {
        double x0[3], p0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x0[c] = xv[e + c];
          p0[c] = phv[e + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) xv[e + c] = fma(alpha, p0[c], x0[c]);
      } else {
        double x0[3], p0[3], h0[3], t0[3], s0[3], q0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x0[c] = xv[e + c];
          p0[c] = phv[e + c];
          h0[c] = shv[e + c];
          t0[c] = tv[e + c];
          s0[c] = sv[e + c];
          q0[c] = rhv[e + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xv[e + c] = fma(alpha, p0[c], fma(omega, h0[c], x0[c]));
          const double rr = fma(-omega, t0[c], s0[c]);
          rv[e + c] = rr;
          acc[0] = fma(rr, rr, acc[0]);
          acc[1] = fma(q0[c], rr, acc[1]);
        }
      }
    }
  }
  double tot[2];
  if (red_end<2>(acc, rs_, S, lt, S.ntiles, tot) && (threadIdx.x & 31) == 0) {
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
// order (zeros on a failed solve).
__global__ void __launch_bounds__(256, 8) k_finish(Batch B) {
  __shared__ RedShared<1> rs_;
  red_begin<1>(rs_);
  OPM_TILE_S(B, S, lt);
  if (S.skip) return;
  const int status = S.st->status;
  const bool ok = (status == OPM_OK || status == OPM_NOT_CONVERGED) && S.st->error == 0;
  double acc[1] = {0.0};
  const int i = lt * kSpmvRows + threadIdx.x;
  {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    if (ok) row_operator(S, S.x, i, y0, y1, y2);
    if (i < S.n) {
      const int o = S.perm[i];
      if (ok) {
        const double d0 = S.b_in[3ll * o] - y0, d1 = S.b_in[3ll * o + 1] - y1, d2 = S.b_in[3ll * o + 2] - y2;
        acc[0] = fma(d0, d0, fma(d1, d1, fma(d2, d2, acc[0])));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) S.x_out[3ll * o + c] = ok ? S.x[3ll * i + c] : 0.0;
    }
  }
  double tot[1];
  if (red_end<1>(acc, rs_, S, lt, S.ntiles_s, tot) && (threadIdx.x & 31) == 0) {
    DevState *st = S.st;
    st->relres = !ok ? nan("") : (st->n0 > 0.0 ? sqrt(tot[0]) / st->n0 : 0.0);
  }
}

// y = A x in the caller's order (x already permuted into w).
__global__ void __launch_bounds__(256, 8) k_spmv_plain(Batch B) {
  OPM_TILE_S(B, S, lt);
  const int i = lt * kSpmvRows + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_operator(S, S.w, i, y0, y1, y2);
  if (i < S.n) {
    const int o = S.perm[i];
    S.x_out[3ll * o] = y0;
    S.x_out[3ll * o + 1] = y1;
    S.x_out[3ll * o + 2] = y2;
  }
}

// w[i] = b_in[perm[i]] (caller's order -> schedule order).
__global__ void __launch_bounds__(256, 6) k_gather(Batch B) {
  OPM_TILE(B, S, lt);
  OPM_TILE_ROWS(i, lt) {
    if (i < S.n) {
      const int o = S.perm[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) S.w[3ll * i + c] = S.b_in[3ll * o + c];
    }
  }
}

// x_out[perm[i]] = t[i] (schedule order -> caller's order).
__global__ void __launch_bounds__(256, 6) k_scatter(Batch B) {
  OPM_TILE(B, S, lt);
  OPM_TILE_ROWS(i, lt) {
    if (i < S.n) {
      const int o = S.perm[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) S.x_out[3ll * o + c] = S.t[3ll * i + c];
    }
  }
}

// ------------------------------------------------------------ control

// Clears the error words of every system and the grid barrier before a
// factorisation or a standalone preconditioner application.
__global__ void k_begin_factor(Batch B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) B.bar[0] = 0;
  if (s < B.nsys && !B.sys[s].skip) {
    DevState *st = B.sys[s].st;
    st->ferror = 0;
    st->error = 0;
    st->err_row = 0x7fffffff;
  }
}

// After a factorisation: a recorded error becomes the factorisation error.
__global__ void k_end_factor(Batch B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B.nsys && !B.sys[s].skip) {
    DevState *st = B.sys[s].st;
    if (st->error != 0) st->ferror = st->error;
  }
}

// Outcome of every system for the host.
__global__ void k_results(Batch B, Result *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B.nsys) {
    const DevState *st = B.sys[s].st;
    Result r;
    r.status = st->error != 0 ? st->error : st->status;
    r.iters = st->iters;
    r.err_row = st->err_row;
    r.pad = 0;
    r.relres = st->relres;
    out[s] = r;
  }
}

// While-loop condition of the solve graph: continue while a system runs.
__global__ void k_loop_cond(Batch B, cudaGraphConditionalHandle h) {
  pdl_enter();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < B.nsys; s += blockDim.x)
    if (!B.sys[s].skip && running(B.sys[s].st)) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// Grid-wide barrier (the cooperative sweep and factorisation launches).

// Grid-wide barrier of a cooperative launch with a bounded wait.  On timeout
// it records OPM_ERR_TIMEOUT in every system and lets the CTA continue;
// after a timeout later barriers do not wait.  The CTA numbered skip_cta (a
// test hook, normally -1) never arrives, so the others' waits run out.
__device__ __forceinline__ void grid_sync(const Batch &B, bool &timed_out) {
  __syncthreads();
  __shared__ int to;
  if (threadIdx.x == 0) {
    to = timed_out ? 1 : 0;
    if ((int)blockIdx.x != B.skip_cta) {
      uint32_t *count = B.bar, *genp = B.bar + 32;
      const uint32_t gen = ld_acquire(genp);
      __threadfence();
      if (atomicAdd(count, 1u) == gridDim.x - 1) {
        *count = 0;
        __threadfence();
        st_release(genp, gen + 1);
      } else if (!to) {
        const uint64_t t0 = gtimer();
        for (uint32_t it = 0;; ++it) {
          if (ld_acquire(genp) != gen) break;
          __nanosleep(32);
          if ((it & 63u) == 63u && gtimer() - t0 > B.spin_limit_ns) {
            for (int s = 0; s < B.nsys; ++s) atomicCAS(&B.sys[s].st->error, 0, (int32_t)OPM_ERR_TIMEOUT);
            to = 1;
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  timed_out = to != 0;
}

}  // namespace opm
