// Kernels of restarted GMRES(m) (OPM's other Krylov solver, Section 2):
// products with the system operator in the schedule's order, and the
// vector work of the Arnoldi process with classical Gram-Schmidt applied
// twice: all projections of a pass in one launch (partial sums per 256-row
// tile, then a fixed-order reduction), the corrections in another.  The
// scalar part (Hessenberg column, Givens rotations, the small triangular
// solve) runs on the host in FP64, as in the oracle.
#pragma once

#include "kernels.cuh"

namespace opm {

constexpr int kGmMaxVec = 65;  // restart length <= 64, plus one vector

// y = A x - wells (schedule order), one row per thread over 256-row tiles.
__global__ void __launch_bounds__(256) k_gm_operator(Batch B, const double *x, double *y) {
  const Sys &S = B.sys[0];
  const int i = blockIdx.x * kSpmvRows + threadIdx.x;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  row_operator(S, x, i, y0, y1, y2);
  if (i < S.n) {
    y[3ll * i] = y0;
    y[3ll * i + 1] = y1;
    y[3ll * i + 2] = y2;
  }
}

// part[tile][q] = sum over the tile's entries of V_q . w, q < nv (V_q at
// V + q * stride): per row, then a warp butterfly, then the warps in order.
__global__ void __launch_bounds__(256) k_gm_dots(int64_t n3, const double *V, int64_t stride, int nv,
                                                 const double *w, double *part) {
  __shared__ double sm[kGmMaxVec][8];
  const int64_t e0 = (int64_t)blockIdx.x * 3 * kSpmvRows + 3 * threadIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double w0 = 0.0, w1 = 0.0, w2 = 0.0;
  if (e0 + 2 < n3 + 0) {
    w0 = __ldcg(w + e0);
    w1 = __ldcg(w + e0 + 1);
    w2 = __ldcg(w + e0 + 2);
  }
  for (int q = 0; q < nv; ++q) {
    double d[1] = {0.0};
    if (e0 + 2 < n3) {
      const double *v = V + q * stride + e0;
      d[0] = fma(__ldcg(v + 2), w2, fma(__ldcg(v + 1), w1, __ldcg(v) * w0));
    }
    warp_sum<1>(d);
    if (lane == 0) sm[q][wp] = d[0];
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) acc += sm[threadIdx.x][k];
    part[(int64_t)blockIdx.x * kGmMaxVec + threadIdx.x] = acc;
  }
}

// out[q] = sum over tiles (in a fixed order) of part[tile][q]; one CTA per q.
__global__ void __launch_bounds__(256) k_gm_reduce(const double *part, int ntiles, double *out) {
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

// mode 0: w -= sum_q coef[q] V_q; 1: w = sum_q coef[q] V_q (q ascending).
__global__ void __launch_bounds__(256) k_gm_combine(int64_t n3, const double *V, int64_t stride, int nv,
                                                    const double *coef, double *w, int mode) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nv; ++q) acc = fma(__ldcg(coef + q), __ldcg(V + q * stride + e), acc);
    w[e] = mode == 0 ? w[e] - acc : acc;
  }
}

// out = w / sqrt(*nrm2) (zero when *nrm2 == 0), or w / beta when nrm2 is null.
__global__ void __launch_bounds__(256) k_gm_scale(int64_t n3, const double *w, const double *nrm2, double beta,
                                                  double *out) {
  const double d = nrm2 ? sqrt(__ldcg(nrm2)) : beta;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = d != 0.0 ? w[e] / d : 0.0;
}

// out = a - b (mode 0), out += a (mode 1)
__global__ void __launch_bounds__(256) k_gm_vec(int64_t n3, const double *a, const double *b, double *out,
                                                int mode) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = mode == 0 ? a[e] - b[e] : out[e] + a[e];
}

}  // namespace opm
