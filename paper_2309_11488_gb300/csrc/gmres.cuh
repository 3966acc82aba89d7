// Kernels of restarted GMRES(m) (OPM's other Krylov solver, Section 2):
// products with the system operator in the schedule's order, and the
// vector work of the Arnoldi process with classical Gram-Schmidt applied
// twice: all projections of a pass in one launch (partial sums per tile,
// then a fixed-order reduction), the corrections in another.  The scalar
// part (Hessenberg column, Givens rotations, the small triangular solve, the
// restart test) runs in FP64 on the device, in one thread, in the oracle's
// order; the whole solve is one graph launch whose Arnoldi steps are the
// body of a device-side while loop.
#pragma once

#include "kernels.cuh"

namespace opm {

constexpr int kGmMaxVec = 65;  // restart length <= 64, plus one vector

// y = A x - wells (schedule order), one row per thread over 256-row tiles.
// The Arnoldi step's product v = A t right after t = inv(M) w
// (APPLIED: row_operator_applied with w as the application's input, tiles
// in the runner's longest-first order).
template <bool APPLIED>
__global__ void __launch_bounds__(256) k_gm_operator(Batch B, const double *x, double *y) {
  const Sys &S = B.sys[0];
  const int i = (APPLIED ? B.tiles_s[blockIdx.x].y : (int)blockIdx.x) * kSpmvRows + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  if (APPLIED) row_operator_applied<true>(S, x, S.w, i, y0, y1, y2);
  else row_operator(S, x, i, y0, y1, y2);
  if (i < S.n) {
    y[3ll * i] = y0;
    y[3ll * i + 1] = y1;
    y[3ll * i + 2] = y2;
  }
}

// ------------------------------------------------------------------
// Device-side control of one GMRES(m) solve (the oracle's steps in its
// order).  sel arguments pick a vector from the state: the Arnoldi column
// j (0), or a fixed one (1).

struct GmState {
  double tol, n0, beta, nrm2;  // nrm2: the last ||w||^2 or ||r||^2
  double relres;
  int32_t m, maxit, j, k;      // restart length, step limit, column, steps taken
  int32_t status;              // kRunning while the solve goes on, then an opm_status
  int32_t conv;                // the cycle ended by the stopping rule
  int32_t update;              // the closing cycle updates x (not after a breakdown)
  int32_t pad;
  double h1[kGmMaxVec], h2[kGmMaxVec], y[kGmMaxVec];
  double cs[kGmMaxVec], sn[kGmMaxVec], g[kGmMaxVec];
  double H[kGmMaxVec * kGmMaxVec];  // H[i * kGmMaxVec + c], (m + 1) x m used
};

__device__ __forceinline__ int gm_nv(const GmState *gs, int sel) { return sel == 0 ? gs->j + 1 : 1; }

// The Gram-Schmidt kernels work on tiles of 256 R rows, R rows per thread
// (rows t, t + 256, ... of the tile): a thread sums its rows before the
// warp reduces, and the warp reduces eight projections at once
// (warp_sum8_split), since a butterfly per value costs the FP64 pipe as much
// per thread as the dots themselves.  With one row per thread a projection
// pass took 15.5 us per basis vector at the 949,871-cell system, bound by
// that pipe.  The host picks R so that the tiles fill whole rounds of the
// SMs (gm_rows_per_thread).

// Sums each of v[0..7] over the 32 lanes of the warp with 9 shuffles and
// additions per lane instead of 40: three halving exchanges (a lane keeps
// half of its values and adds its partner's copies of them) leave lane l
// with value l >> 2 summed over 8 lanes, and two butterfly steps finish it.
// Returns value (lane >> 2)'s sum; every step adds the same two numbers in
// both partners, so all four lanes holding a value hold the same bits.
__device__ __forceinline__ double warp_sum8_split(const double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  double u[4], t[2];
  bool hi = lane & 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double keep = hi ? v[i + 4] : v[i], send = hi ? v[i] : v[i + 4];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  hi = lane & 8;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double keep = hi ? u[i + 2] : u[i], send = hi ? u[i] : u[i + 2];
    t[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  hi = lane & 4;
  double s = (hi ? t[1] : t[0]) + __shfl_xor_sync(0xffffffffu, hi ? t[0] : t[1], 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

// The partial projections V_q . x over this thread's R rows (x[k] = its
// entries of row k), reduced over the warp in chunks of eight and stored
// to sm[q][warp] for q < nv.
template <int R>
__device__ __forceinline__ void gm_project(int64_t n3, const double *V, int64_t stride, int64_t b0, int nv,
                                           const double (&x)[R][3], double (*sm)[8]) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int q0 = 0; q0 < nv; q0 += 8) {
    double d[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      d[u] = 0.0;
      if (q0 + u < nv) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int64_t e = b0 + 3 * 256 * k;
          if (e + 2 < n3) {
            const double *v = V + (q0 + u) * stride + e;
            d[u] = fma(__ldcg(v + 2), x[k][2], fma(__ldcg(v + 1), x[k][1], fma(__ldcg(v), x[k][0], d[u])));
          }
        }
      }
    }
    const double s = warp_sum8_split(d);
    if ((lane & 3) == 0 && q0 + (lane >> 2) < nv) sm[q0 + (lane >> 2)][wp] = s;
  }
}

// part[tile][q] = V_q . w for q < nv (sel 0: the columns 0..j; sel 1: V = w
// itself, nv = 1), as k_gm_dots.
template <int R>
__global__ void __launch_bounds__(256) k_gm_dots_s(int64_t n3, const double *V, int64_t stride, const GmState *gs,
                                                   int sel, const double *w, double *part) {
  __shared__ double sm[kGmMaxVec][8];
  const int nv = gm_nv(gs, sel);
  const int64_t b0 = (int64_t)blockIdx.x * 3 * 256 * R + 3 * threadIdx.x;
  double x[R][3];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int64_t e = b0 + 3 * 256 * k;
    const bool in = e + 2 < n3;
    x[k][0] = in ? __ldcg(w + e) : 0.0;
    x[k][1] = in ? __ldcg(w + e + 1) : 0.0;
    x[k][2] = in ? __ldcg(w + e + 2) : 0.0;
  }
  gm_project<R>(n3, V, stride, b0, nv, x, sm);
  __syncthreads();
  if (threadIdx.x < nv) {
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) acc += sm[threadIdx.x][k];
    part[(int64_t)blockIdx.x * kGmMaxVec + threadIdx.x] = acc;
  }
}

// out[q] = sum over tiles of part[tile][q], q < nv; one CTA per q (a grid of
// kGmMaxVec CTAs, the ones past nv return).
__global__ void __launch_bounds__(256) k_gm_reduce_s(const double *part, int ntiles, const GmState *gs, int sel,
                                                     double *out) {
  if ((int)blockIdx.x >= gm_nv(gs, sel)) return;
  __shared__ double sm[8];
  const int q = blockIdx.x;
  double acc[1] = {0.0};
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) acc[0] += __ldcg(part + (int64_t)t * kGmMaxVec + q);
  warp_sum<1>(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc[0];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sm[k];
    out[q] = s;
  }
}

// A Gram-Schmidt correction fused with what follows it, over the tiles of
// k_gm_dots_s: w -= sum_{q <= j} coef[q] V_q, then (NEXT_DOTS) the partial
// projections V_q . w of the corrected w for q <= j, or (!NEXT_DOTS) the
// partial ||w||^2.  Each entry's correction is the same expression as in
// k_gm_combine_s and each partial projection the same as in k_gm_dots_s, so
// the results are those of the separate kernels, with one pass over V and w
// fewer.
template <int R, bool NEXT_DOTS>
__global__ void __launch_bounds__(256) k_gm_correct_s(int64_t n3, const double *V, int64_t stride, const GmState *gs,
                                                      const double *coef, double *w, double *part) {
  __shared__ double c[kGmMaxVec];
  __shared__ double sm[kGmMaxVec][8];
  const int nv = gs->j + 1;
  for (int q = threadIdx.x; q < nv; q += blockDim.x) c[q] = coef[q];
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * 3 * 256 * R + 3 * threadIdx.x;
  double x[R][3];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int64_t e = b0 + 3 * 256 * k;
    x[k][0] = x[k][1] = x[k][2] = 0.0;
    if (e + 2 < n3) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int q = 0; q < nv; ++q) {
        const double *v = V + q * stride + e;
        a0 = fma(c[q], __ldcg(v), a0);
        a1 = fma(c[q], __ldcg(v + 1), a1);
        a2 = fma(c[q], __ldcg(v + 2), a2);
      }
      x[k][0] = w[e] - a0;
      x[k][1] = w[e + 1] - a1;
      x[k][2] = w[e + 2] - a2;
      w[e] = x[k][0];
      w[e + 1] = x[k][1];
      w[e + 2] = x[k][2];
    }
  }
  if (NEXT_DOTS) {
    gm_project<R>(n3, V, stride, b0, nv, x, sm);
  } else {
    double d[1] = {0.0};
#pragma unroll
    for (int k = 0; k < R; ++k)
      d[0] = fma(x[k][2], x[k][2], fma(x[k][1], x[k][1], fma(x[k][0], x[k][0], d[0])));
    warp_sum<1>(d);
    if ((threadIdx.x & 31) == 0) sm[0][threadIdx.x >> 5] = d[0];
  }
  __syncthreads();
  const int nd = NEXT_DOTS ? nv : 1;
  if (threadIdx.x < nd) {
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) acc += sm[threadIdx.x][k];
    part[(int64_t)blockIdx.x * kGmMaxVec + threadIdx.x] = acc;
  }
}

// The Gram-Schmidt kernels for R rows per thread.
struct GmKernels {
  void (*dots)(int64_t, const double *, int64_t, const GmState *, int, const double *, double *);
  void (*correct)(int64_t, const double *, int64_t, const GmState *, const double *, double *, double *);
  void (*correct_norm)(int64_t, const double *, int64_t, const GmState *, const double *, double *, double *);
  int rows;  // rows per tile, 256 R
};

template <int R>
GmKernels gm_kernels_for() {
  return {k_gm_dots_s<R>, k_gm_correct_s<R, true>, k_gm_correct_s<R, false>, 256 * R};
}

// Rows per thread of the Gram-Schmidt kernels for n rows on sms SMs: the one
// of 4, 5, 6 whose tiles give the smallest per-SM share when every SM takes
// whole tiles, the smaller R on ties (more threads per row).  On 152 SMs
// R = 4 up to 155,648 rows, then each of the three in turn (R = 5 at the
// 949,871-cell system); a larger R never wins below 1.2 M rows.
inline GmKernels gm_rows_per_thread(int64_t n, int sms) {
  const GmKernels k[3] = {gm_kernels_for<4>(), gm_kernels_for<5>(), gm_kernels_for<6>()};
  int best = 0;
  int64_t cost = -1;
  for (int i = 0; i < 3; ++i) {
    const int64_t tiles = (n + k[i].rows - 1) / k[i].rows;
    const int64_t c = ((tiles + sms - 1) / sms) * k[i].rows;
    if (cost < 0 || c < cost) cost = c, best = i;
  }
  return k[best];
}

// mode 0: w -= sum_{q <= j} coef[q] V_q (a Gram-Schmidt pass); mode 1:
// w = sum_{q < j} y[q] V_q (the cycle's correction, only when it updates x).
__global__ void __launch_bounds__(256) k_gm_combine_s(int64_t n3, const double *V, int64_t stride, const GmState *gs,
                                                      const double *coef, double *w, int mode) {
  __shared__ double c[kGmMaxVec];
  if (mode == 1 && !gs->update) return;
  const int nv = mode == 0 ? gs->j + 1 : gs->j;
  for (int q = threadIdx.x; q < nv; q += blockDim.x) c[q] = coef[q];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nv; ++q) acc = fma(c[q], __ldcg(V + q * stride + e), acc);
    w[e] = mode == 0 ? w[e] - acc : acc;
  }
}

// sel 0: V_{j+1} = w / sqrt(nrm2) (zero when the norm is); sel 1: V_0 = w /
// beta at the start of a cycle (only while the solve runs).  The new basis
// vector also goes to next, the next Arnoldi step's input.  One thread per
// CTA takes the square root and the reciprocal: at one per thread they cost
// more FP64 issue slots than the pass itself.
__global__ void __launch_bounds__(256) k_gm_scale_s(int64_t n3, const double *w, const GmState *gs, int sel,
                                                    double *V, int64_t stride, double *next) {
  __shared__ double srd;
  if (sel == 1 && gs->status != kRunning) return;
  if (threadIdx.x == 0) {
    const double d = sel == 0 ? sqrt(gs->nrm2) : gs->beta;
    srd = d != 0.0 ? 1.0 / d : 0.0;
  }
  __syncthreads();
  const double rd = srd;
  double *out = V + (sel == 0 ? (int64_t)(gs->j + 1) * stride : 0);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    const double u = w[e] * rd;
    out[e] = u;
    next[e] = u;
  }
}

// dst = src.
__global__ void __launch_bounds__(256) k_gm_copy_s(int64_t n3, const double *src, double *dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// mode 0: out = a - b; mode 1: out += a when the closing cycle updates x;
// mode 2: out = 0 when the solve failed (negative status).
__global__ void __launch_bounds__(256) k_gm_vec_s(int64_t n3, const double *a, const double *b, double *out, int mode,
                                                  const GmState *gs) {
  if (mode == 1 && !gs->update) return;
  if (mode == 2 && gs->status >= 0) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = mode == 0 ? a[e] - b[e] : mode == 1 ? out[e] + a[e] : 0.0;
}

// Start: n0 = ||b||, the stopping threshold, the first cycle's g; the loop
// runs only when there is something to solve.  gs->tol holds rtol on entry.
__global__ void k_gm_init(GmState *gs, cudaGraphConditionalHandle loop) {
  const double n0 = sqrt(gs->nrm2);
  gs->n0 = n0;
  gs->j = 0;
  gs->k = 0;
  gs->conv = 0;
  gs->update = 0;
  if (!isfinite(n0)) gs->status = OPM_ERR_NONFINITE;
  else if (n0 == 0.0) gs->status = OPM_OK;
  else if (gs->maxit == 0) gs->status = OPM_NOT_CONVERGED;
  else gs->status = kRunning;
  gs->tol = gs->tol * n0;
  gs->beta = n0;
  for (int i = 0; i < kGmMaxVec; ++i) gs->g[i] = 0.0;
  gs->g[0] = n0;
  cudaGraphSetConditional(loop, gs->status == kRunning ? 1u : 0u);
}

// One Arnoldi step's scalar part: the Hessenberg column from the two
// Gram-Schmidt passes and the norm, the earlier rotations, the new
// rotation, g, and the end-of-cycle test (stopping rule, restart length,
// step limit); a zero rotation is a breakdown and a non-finite g a failure,
// both ending the solve without an update.  Opens the end-of-cycle branch.
__global__ void k_gm_step(GmState *gs, cudaGraphConditionalHandle cycle_end) {
  const int j = gs->j, m = gs->m;
  constexpr int L = kGmMaxVec;
  double *H = gs->H;
  gs->k += 1;
  for (int i = 0; i <= j; ++i) H[i * L + j] = gs->h1[i] + gs->h2[i];
  const double hn = sqrt(gs->nrm2);
  H[(j + 1) * L + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * L + j], c = H[(i + 1) * L + j];
    H[i * L + j] = gs->cs[i] * a + gs->sn[i] * c;
    H[(i + 1) * L + j] = -gs->sn[i] * a + gs->cs[i] * c;
  }
  const double a = H[j * L + j], c = H[(j + 1) * L + j];
  const double den = sqrt(a * a + c * c);
  bool end = false;
  if (den == 0.0) {
    gs->status = OPM_ERR_BREAKDOWN;
    gs->update = 0;
    end = true;
  } else {
    gs->cs[j] = a / den;
    gs->sn[j] = c / den;
    H[j * L + j] = den;
    H[(j + 1) * L + j] = 0.0;
    gs->g[j + 1] = -gs->sn[j] * gs->g[j];
    gs->g[j] = gs->cs[j] * gs->g[j];
    if (!isfinite(gs->g[j + 1])) {
      gs->status = OPM_ERR_NONFINITE;
      gs->update = 0;
      end = true;
    } else {
      const bool conv = fabs(gs->g[j + 1]) <= gs->tol || hn == 0.0;
      gs->j = j + 1;
      gs->conv = conv;
      end = conv || j + 1 == m || gs->k >= gs->maxit;
      gs->update = end;
    }
  }
  cudaGraphSetConditional(cycle_end, end ? 1u : 0u);
}

// End of a cycle: H y = g by back substitution over the cycle's j columns.
__global__ void k_gm_trisolve(GmState *gs) {
  if (!gs->update) return;
  const int j = gs->j;
  constexpr int L = kGmMaxVec;
  for (int i = j - 1; i >= 0; --i) {
    double acc = gs->g[i];
    for (int l = i + 1; l < j; ++l) acc -= gs->H[i * L + l] * gs->y[l];
    gs->y[i] = acc / gs->H[i * L + i];
  }
}

// After a cycle's update and the residual norm: stop (the stopping rule,
// the step limit, or a failure), or restart with beta = ||r||.
__global__ void k_gm_restart(GmState *gs) {
  if (gs->status == kRunning) {
    if (gs->conv) {
      gs->status = OPM_OK;
    } else if (gs->k >= gs->maxit) {
      gs->status = OPM_NOT_CONVERGED;
    } else {
      const double beta = sqrt(gs->nrm2);
      gs->beta = beta;
      if (beta <= gs->tol) {
        gs->status = OPM_OK;
      } else {
        gs->j = 0;
        for (int i = 0; i < kGmMaxVec; ++i) gs->g[i] = 0.0;
        gs->g[0] = beta;
      }
    }
  }
  gs->update = 0;
  gs->conv = 0;
}

__global__ void k_gm_cond(const GmState *gs, cudaGraphConditionalHandle loop) {
  cudaGraphSetConditional(loop, gs->status == kRunning ? 1u : 0u);
}

// The true residual's norm (relres; NaN after a non-finite failure).
__global__ void k_gm_final(GmState *gs) {
  gs->relres = gs->status == OPM_ERR_NONFINITE ? nan("") : gs->n0 > 0.0 ? sqrt(gs->nrm2) / gs->n0 : 0.0;
}

}  // namespace opm
