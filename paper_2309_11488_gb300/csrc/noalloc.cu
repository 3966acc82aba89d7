// Allocation-free residual entry point.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running inside a simulator's own memory pool or arena (which
// forbids foreign cudaMalloc calls), code called while the caller holds a
// fixed device-memory budget it must not exceed, or code in a process where
// every allocation goes through an allocator the library cannot see.  For
// them, opm_bsr_residual_noalloc computes r = b - A x and the 2-norms
// ||r||_2, ||b||_2 on the caller's own BSR arrays without creating a handle
// and without allocating anything.
//
// Its only scratch (one partial sum pair per 256-row tile, the last-CTA
// counter and a pattern-error word) is the file-scope array below: every GPU
// that loads the library holds these 131,328 bytes until the process exits,
// every call shares them, and they keep the last call's contents.  The
// counter and the error word are cleared at the start of every call.  Calls
// that overlap on the GPU (on two streams, or from two host threads) race on
// the array and give wrong results: serialise them.
//
// The caller's pattern is not validated on the host (that would need a copy
// of it).  The kernel checks what it can before each access: a row whose
// start is negative or whose end lies before its start is taken as empty, a
// column outside [0, nb) is skipped; either sets the error word, the norms
// become NaN and the call returns OPM_ERR_PATTERN.  rowptr[nb] beyond the
// length of colidx and vals cannot be detected without that length: a
// well-formed pattern is the caller's precondition.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/opm_bsr.h"

namespace {

constexpr int kNaTile = 256;                   // rows per CTA
constexpr int kNaMaxTiles = 8192;              // => at most 2,097,152 block rows
constexpr size_t kNaCounterBytes = 256;        // counter and error word, padded to their own lines
constexpr size_t kNaScratchBytes = kNaCounterBytes + sizeof(double) * 2 * kNaMaxTiles;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once
// per device, with that device current, and kept: calls after a
// cudaDeviceReset of that device are not supported, since the reloaded
// module may place the array elsewhere).
opm_status scratch_address(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return OPM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return OPM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return OPM_OK;
}

// True for device (or managed) memory of the current device; host memory
// and another GPU's memory are refused.
bool on_device(const void *p) {
  cudaPointerAttributes at;
  int dev = -1;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// One thread per block row of the caller's BSR matrix (row-major 3x3 blocks):
// r_i = b_i - sum_j A_ij x_j; per-CTA partials of ||r||^2 and ||b||^2 in the
// scratch array; the last CTA sums them in tile order.  Pattern faults that
// can be seen from the row (see the file header) skip the access and set the
// error word; the last CTA then writes NaN norms.
__global__ void __launch_bounds__(kNaTile) k_residual_noalloc(int32_t nb, const int32_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx,
                                                              const double *__restrict__ vals,
                                                              const double *__restrict__ x,
                                                              const double *__restrict__ b, double *__restrict__ r,
                                                              double *__restrict__ norms, unsigned char *scratch) {
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch);
  unsigned int *bad = counter + 1;
  double *partials = reinterpret_cast<double *>(scratch + kNaCounterBytes);
  const int i = blockIdx.x * kNaTile + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < nb) {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    int m0 = rowptr[i], m1 = rowptr[i + 1];
    if (m0 < 0 || m1 < m0) {
      atomicOr(bad, 1u);
      m1 = m0;
    }
    for (int m = m0; m < m1; ++m) {
      const int c = colidx[m];
      if (c < 0 || c >= nb) {
        atomicOr(bad, 1u);
        continue;
      }
      const double *a = vals + 9ll * m;
      const int64_t j = 3ll * c;
      const double x0 = x[j], x1 = x[j + 1], x2 = x[j + 2];
      y0 = fma(a[0], x0, fma(a[1], x1, fma(a[2], x2, y0)));
      y1 = fma(a[3], x0, fma(a[4], x1, fma(a[5], x2, y1)));
      y2 = fma(a[6], x0, fma(a[7], x1, fma(a[8], x2, y2)));
    }
    const double b0 = b[3ll * i], b1 = b[3ll * i + 1], b2 = b[3ll * i + 2];
    const double d0 = b0 - y0, d1 = b1 - y1, d2 = b2 - y2;
    r[3ll * i] = d0;
    r[3ll * i + 1] = d1;
    r[3ll * i + 2] = d2;
    rr = fma(d0, d0, fma(d1, d1, d2 * d2));
    bb = fma(b0, b0, fma(b1, b1, b2 * b2));
  }
  __shared__ double sm[2][kNaTile / 32];
  __shared__ int amlast;
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[0][threadIdx.x >> 5] = rr;
    sm[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kNaTile / 32; ++w) {
      a += sm[0][w];
      c += sm[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = c;
    __threadfence();
    amlast = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!amlast || threadIdx.x != 0) return;
  __threadfence();
  double a = 0.0, c = 0.0;
  for (unsigned t = 0; t < gridDim.x; ++t) {
    a += __ldcg(partials + 2 * t);
    c += __ldcg(partials + 2 * t + 1);
  }
  const bool faulty = __ldcg(bad) != 0u;
  norms[0] = faulty ? nan("") : sqrt(a);
  norms[1] = faulty ? nan("") : sqrt(c);
  *counter = 0;
}

}  // namespace

extern "C" opm_status opm_bsr_residual_noalloc(int32_t nb, const int32_t *rowptr, const int32_t *colidx,
                                               const double *vals, const double *x, const double *b,
                                               double *r, double *norms, void *stream) {
  if (nb < 0 || nb > kNaMaxTiles * kNaTile) return OPM_ERR_ARG;  // beyond the scratch capacity
  if (!norms || !on_device(norms)) return OPM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nb == 0) {
    if (cudaMemsetAsync(norms, 0, 2 * sizeof(double), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return OPM_ERR_CUDA;
    }
    return OPM_OK;
  }
  if (!on_device(rowptr) || !on_device(colidx) || !on_device(vals) || !on_device(x) || !on_device(b) ||
      !on_device(r))
    return OPM_ERR_ARG;
  unsigned char *scratch = nullptr;
  opm_status s = scratch_address(&scratch);
  if (s != OPM_OK) return s;
  const int tiles = (nb + kNaTile - 1) / kNaTile;
  if (cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
    cudaGetLastError();
    return OPM_ERR_CUDA;
  }
  k_residual_noalloc<<<tiles, kNaTile, 0, st>>>(nb, rowptr, colidx, vals, x, b, r, norms, scratch);
  unsigned int bad = 0;  // host copy of the error word (a pageable copy allocates no device memory)
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, scratch + sizeof(unsigned int), sizeof bad, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return OPM_ERR_CUDA;
  }
  return bad ? OPM_ERR_PATTERN : OPM_OK;
}
