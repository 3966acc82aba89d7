// Host driver and C ABI of the GB300 BSR ILU0-BiCGStab library.
//
// A handle owns the schedule-ordered device copy of the matrix, its ILU0
// factors, the Krylov vectors and a CUDA graph holding `chunk` BiCGStab
// iterations (5 kernel nodes each).  A solve is: one setup launch, graph
// launches until the device status word leaves "running" (the host reads it
// once per chunk), one finishing launch for the true residual.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"

using namespace opm;

struct opm_solver {
  Analysis an;
  opm_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int32_t n = 0, nslices = 0, ntiles = 0;
  int64_t nnzb = 0;
  bool fp32 = false;
  Sys sys{};
  int grid_apply = 1, grid_factor = 1;
  int chunk = 8;
  cudaGraphExec_t chunk_exec = nullptr;
  int chunk_launches = 0;  // kernel nodes in the chunk graph
  bool cooperative = false;  // sweeps as one cooperative launch
  DevState *h_state = nullptr;  // pinned
  std::vector<void *> allocs;
  double *vals_stage = nullptr;   // caller's values when given from host
  double *vec_in = nullptr, *vec_out = nullptr;  // caller-order staging
  int64_t dev_bytes = 0;
  int32_t last_err_row = -1;
  bool factors_ok = false;
  opm_timing timing{};
  cudaEvent_t ev[6] = {};
  std::vector<cudaEvent_t> kev;  // per-kernel events inside the graph (profiling)
};

namespace {

thread_local int32_t t_create_err_row = -1;  // row of this thread's last failed create

const char *const kStatusText[] = {"ok",
                                   "not converged within maxit",
                                   "invalid argument",
                                   "invalid sparsity pattern",
                                   "missing diagonal block",
                                   "singular pivot block in ILU0",
                                   "BiCGStab breakdown",
                                   "non-finite right-hand side",
                                   "out of device memory",
                                   "device wait timed out",
                                   "CUDA error"};

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      fprintf(stderr, "opm_bsr: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? OPM_ERR_OOM : OPM_ERR_CUDA; \
    }                                                 \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
opm_status dalloc(opm_solver *h, T **p, size_t count) {
  *p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? OPM_ERR_OOM : OPM_ERR_CUDA;
  }
  h->allocs.push_back(*p);
  h->dev_bytes += (int64_t)bytes;
  return OPM_OK;
}

template <typename T>
opm_status upload(opm_solver *h, T **p, const std::vector<T> &v) {
  opm_status s = dalloc(h, p, v.size());
  if (s != OPM_OK) return s;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return OPM_OK;
}

int blocks_for(int n) { return std::max(1, (n + kTileRows - 1) / kTileRows); }

// Sweep kernels are launched cooperatively: the launch fails instead of
// starting when its CTAs cannot all be resident at once.
template <typename... P, typename... A>
cudaError_t launch_coop(void (*kern)(P...), int grid, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// CTAs of 8 warps covering the slices of rows [r0, r1)
int phase_blocks(int r0, int r1) { return (((r1 - 1) >> 5) - (r0 >> 5) + 1 + 7) / 8; }

// Schedules with at most this many phases run one launch per phase; more
// phases run as one cooperative launch with grid barriers.
constexpr int kMaxPhaseLaunches = 1024;

template <typename TF>
int launch_factor(opm_solver *h, const double *vals_user, cudaStream_t st) {
  const Sys &S = h->sys;
  if (h->cooperative) {
    launch_coop(k_factor<TF>, h->grid_factor, st, S, vals_user);
    return 1;
  }
  const std::vector<int32_t> &pp = h->an.phase_ptr;
  for (int p = 0; p < S.nphases; ++p)
    k_factor_phase<TF><<<phase_blocks(pp[p], pp[p + 1]), 256, 0, st>>>(S, pp[p], pp[p + 1], vals_user);
  return S.nphases;
}

template <typename TF, int MODE>
int launch_apply(opm_solver *h, const double *in, double *out, cudaStream_t st) {
  const Sys &S = h->sys;
  if (h->cooperative) {
    launch_coop(k_apply<TF, MODE>, h->grid_apply, st, S, in, out);
    return 1;
  }
  const std::vector<int32_t> &pp = h->an.phase_ptr;
  const int np = S.nphases;
  for (int p = 0; p < np; ++p)
    k_fwd_phase<TF, MODE><<<phase_blocks(pp[p], pp[p + 1]), 256, 0, st>>>(S, pp[p], pp[p + 1], p == np - 1, in,
                                                                            out);
  for (int p = np - 2; p >= 0; --p)
    k_bwd_phase<TF, MODE><<<phase_blocks(pp[p], pp[p + 1]), 256, 0, st>>>(S, pp[p], pp[p + 1], out);
  return 2 * np - 1;
}

template <int MODE>
int launch_apply_p(opm_solver *h, const double *in, double *out, cudaStream_t st) {
  return h->fp32 ? launch_apply<float, MODE>(h, in, out, st) : launch_apply<double, MODE>(h, in, out, st);
}

// One BiCGStab iteration: 5 kernels.  With ev (6 events), the kernels are
// bracketed by event-record nodes (external records, so that they are real
// graph nodes rather than capture-internal dependencies) for per-kernel
// timing.
int launch_iteration(opm_solver *h, cudaStream_t st, cudaEvent_t *ev) {
  const int nb = h->ntiles;
  auto mark = [&](int q) {
    if (ev) cudaEventRecordWithFlags(ev[q], st, cudaEventRecordExternal);
  };
  int launches = 3;
  mark(0);
  launches += launch_apply_p<kModeP>(h, nullptr, nullptr, st);
  mark(1);
  k_spmv_v<<<nb, 1024, 0, st>>>(h->sys);
  mark(2);
  launches += launch_apply_p<kModeS>(h, nullptr, nullptr, st);
  mark(3);
  k_spmv_t<<<nb, 1024, 0, st>>>(h->sys);
  mark(4);
  k_update<<<nb, 256, 0, st>>>(h->sys);
  mark(5);
  return launches;
}

const int kIterKernel[5] = {OPM_KERNEL_APPLY, OPM_KERNEL_SPMV, OPM_KERNEL_APPLY, OPM_KERNEL_SPMV,
                            OPM_KERNEL_UPDATE};

void add_kernel_time(opm_solver *h, int kind, cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
    h->timing.kernel_ms[kind] += ms;
    h->timing.kernel_count[kind] += 1;
  } else {
    cudaGetLastError();
  }
}

// Clears the error word and the grid-barrier counter before a sweep launch
// that does not follow k_setup.
__global__ void k_begin_factor(DevState *st) {
  st->error = 0;
  st->err_row = INT_MAX;
  st->bar_count = 0;
}

// Largest co-resident grid of sweep CTAs for a kernel, capped by the work
// (one slice per warp).
template <typename K>
int resident_grid(K kernel, int device, int items) {
  int sms = 1, occ = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kSweepThreads, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int warps = kSweepThreads / 32;
  int want = std::max(1, (items + warps - 1) / warps);
  return std::max(1, std::min(sms * occ, want));
}

// The sweep grids need only as many warps as the largest phase has slices:
// fewer CTAs make the grid barrier cheaper.
int max_phase_slices(const Analysis &an) {
  int m = 1;
  for (size_t p = 0; p + 1 < an.phase_ptr.size(); ++p) {
    const int r0 = an.phase_ptr[p], r1 = an.phase_ptr[p + 1];
    m = std::max(m, (r1 - 1) / kWarp - r0 / kWarp + 1);
  }
  return m;
}

template <typename TF>
int apply_grid(int device, int slices) {
  int g = resident_grid(k_apply<TF, kModeP>, device, slices);
  g = std::min(g, resident_grid(k_apply<TF, kModeS>, device, slices));
  return std::min(g, resident_grid(k_apply<TF, kModePlain>, device, slices));
}

opm_status build_graph(opm_solver *h) {
  cudaStream_t cap;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    h->chunk_launches = 0;
    for (int it = 0; it < h->chunk; ++it)
      h->chunk_launches += launch_iteration(h, cap, h->kev.empty() ? nullptr : &h->kev[6 * it]);
    e = cudaStreamEndCapture(cap, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->chunk_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    fprintf(stderr, "opm_bsr: graph capture failed: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
    return OPM_ERR_CUDA;
  }
  return OPM_OK;
}

opm_status read_state(opm_solver *h) {
  CK(cudaMemcpyAsync(h->h_state, h->sys.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OPM_OK;
}

// Copies a caller vector of 3n doubles to device staging when it is host
// memory; returns the device pointer to read from.
opm_status stage_in(opm_solver *h, const double *src, const double **dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return OPM_OK;
  }
  CK(cudaMemcpyAsync(h->vec_in, src, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
  *dev = h->vec_in;
  return OPM_OK;
}

opm_status factor_impl(opm_solver *h, const double *vals) {
  const double *dv = nullptr;
  if (vals) {
    if (is_device_ptr(vals)) {
      dv = vals;
    } else {
      if (!h->vals_stage) {
        opm_status s = dalloc(h, &h->vals_stage, 9 * (size_t)h->nnzb);
        if (s != OPM_OK) return s;
      }
      CK(cudaMemcpyAsync(h->vals_stage, vals, sizeof(double) * 9 * (size_t)h->nnzb, cudaMemcpyHostToDevice,
                         h->stream));
      dv = h->vals_stage;
    }
  }
  h->factors_ok = false;
  if (h->n == 0) {
    h->factors_ok = true;
    return OPM_OK;
  }
  k_begin_factor<<<1, 1, 0, h->stream>>>(h->sys.st);
  CK(cudaEventRecord(h->ev[4], h->stream));
  const int nl = h->fp32 ? launch_factor<float>(h, dv, h->stream) : launch_factor<double>(h, dv, h->stream);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev[5], h->stream));
  h->timing.launches += 1 + nl;
  opm_status s = read_state(h);
  if (s != OPM_OK) return s;
  cudaEventElapsedTime(&h->timing.factor_ms, h->ev[4], h->ev[5]);
  if (h->opt.profile_kernels) add_kernel_time(h, OPM_KERNEL_FACTOR, h->ev[4], h->ev[5]);
  if (h->h_state->error != 0) {
    int32_t r = h->h_state->err_row;
    h->last_err_row = (r >= 0 && r < h->n) ? h->an.perm[r] : -1;
    return (opm_status)h->h_state->error;
  }
  h->factors_ok = true;
  return OPM_OK;
}

}  // namespace

extern "C" {

void opm_options_default(opm_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->schedule = OPM_SCHED_AUTO;
  opt->precision = OPM_PREC_FP64;
  opt->stream = nullptr;
  opt->chunk = 0;
  opt->spin_limit_us = 0;
  opt->debug_skip_item = -1;
}

const char *opm_status_str(opm_status s) {
  int v = (int)s;
  if (v == 0) return kStatusText[0];
  if (v == 1) return kStatusText[1];
  if (v <= -1 && v >= -9) return kStatusText[1 - v];
  return "unknown status";
}

void opm_destroy(opm_handle h) {
  if (!h) return;
  if (!h->allocs.empty()) cudaStreamSynchronize(h->stream);
  if (h->chunk_exec) cudaGraphExecDestroy(h->chunk_exec);
  for (void *p : h->allocs) cudaFree(p);
  if (h->h_state) cudaFreeHost(h->h_state);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : h->kev)
    if (e) cudaEventDestroy(e);
  delete h;
}

opm_status opm_bsr_create(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                          const opm_options *opt, opm_handle *out) {
  if (!out) return OPM_ERR_ARG;
  *out = nullptr;
  t_create_err_row = -1;
  if (nb < 0 || !rowptr || (nb > 0 && (!colidx || !vals))) return OPM_ERR_ARG;
  opm_options o;
  opm_options_default(&o);
  if (opt) o = *opt;
  if (o.schedule < OPM_SCHED_AUTO || o.schedule > OPM_SCHED_COLOUR) return OPM_ERR_ARG;
  if (o.precision != OPM_PREC_FP64 && o.precision != OPM_PREC_FP32_FACTORS) return OPM_ERR_ARG;
  if (o.chunk < 0 || o.spin_limit_us < 0) return OPM_ERR_ARG;
  if (o.sweep_launch < OPM_SWEEP_AUTO || o.sweep_launch > OPM_SWEEP_COOPERATIVE) return OPM_ERR_ARG;

  opm_solver *h = new (std::nothrow) opm_solver();
  if (!h) return OPM_ERR_OOM;
  h->opt = o;
  h->stream = (cudaStream_t)o.stream;
  h->fp32 = o.precision == OPM_PREC_FP32_FACTORS;
  h->chunk = o.chunk > 0 ? o.chunk : 8;
  auto fail = [&](opm_status s) {
    opm_destroy(h);
    return s;
  };

  // ---- pattern on the host for the analysis
  std::vector<int32_t> hrp, hci;
  const int32_t *rp = rowptr, *ci = colidx;
  if (is_device_ptr(rowptr)) {
    hrp.resize((size_t)nb + 1);
    if (cudaMemcpy(hrp.data(), rowptr, sizeof(int32_t) * hrp.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(OPM_ERR_CUDA);
    rp = hrp.data();
  }
  const int64_t nnzb = rp[nb];
  if (nnzb < 0) return fail(OPM_ERR_PATTERN);
  if (nb > 0 && is_device_ptr(colidx)) {
    hci.resize((size_t)nnzb);
    if (cudaMemcpy(hci.data(), colidx, sizeof(int32_t) * hci.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(OPM_ERR_CUDA);
    ci = hci.data();
  }
  int32_t err_row = -1;
  opm_status s = analyse(nb, rp, ci, o.schedule, h->an, &err_row);
  t_create_err_row = err_row;
  if (s != OPM_OK) return fail(s);
  // ---- CUDA resources (after the host checks, which need no device)
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_CUDA);
  }
  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return fail(OPM_ERR_CUDA);
    }
  if (cudaMallocHost((void **)&h->h_state, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_OOM);
  }
  Analysis &an = h->an;
  h->n = nb;
  h->nnzb = nnzb;
  h->nslices = (nb + kWarp - 1) / kWarp;
  h->ntiles = blocks_for(nb);

  // ---- device buffers
  Sys &S = h->sys;
  S.n = nb;
  S.nslices = h->nslices;
  S.u_off = 9 * an.nnz_l;
  S.d_off = an.d_off;
  S.spin_limit_ns = (uint64_t)(o.spin_limit_us > 0 ? o.spin_limit_us : 2000000) * 1000ull;
  S.skip_cta = o.debug_skip_item;
  int32_t *p_perm, *p_arp, *p_acol, *p_asrc, *p_lrp, *p_lcol, *p_urp, *p_ucol, *p_upd;
  int32_t *p_ph;
  int64_t *p_adst, *p_ud, *p_us;
#define UP(ptr, vec) \
  if ((s = upload(h, &ptr, vec)) != OPM_OK) return fail(s)
  UP(p_perm, an.perm);
  UP(p_arp, an.a_rowptr);
  UP(p_acol, an.a_col);
  UP(p_asrc, an.a_src);
  UP(p_adst, an.a_dst);
  UP(p_lrp, an.l_rowptr);
  UP(p_lcol, an.l_col);
  UP(p_urp, an.u_rowptr);
  UP(p_ucol, an.u_col);
  UP(p_upd, an.upd_ptr);
  UP(p_ud, an.upd_dst);
  UP(p_us, an.upd_src);
  UP(p_ph, an.phase_ptr);
#undef UP
  S.phase_ptr = p_ph;
  S.nphases = (int32_t)an.phase_ptr.size() - 1;
  S.perm = p_perm;
  S.a_rp = p_arp;
  S.a_col = p_acol;
  S.a_src = p_asrc;
  S.a_dst = p_adst;
  S.l_rp = p_lrp;
  S.l_col = p_lcol;
  S.u_rp = p_urp;
  S.u_col = p_ucol;
  S.upd_ptr = p_upd;
  S.upd_dst = p_ud;
  S.upd_src = p_us;
  if ((s = dalloc(h, &S.a_val, 9 * (size_t)nnzb)) != OPM_OK) return fail(s);
  if (h->fp32) {
    float *lu;
    if ((s = dalloc(h, &lu, (size_t)an.lu_vals)) != OPM_OK) return fail(s);
    S.lu = lu;
    float *y;
    if ((s = dalloc(h, &y, 3 * (size_t)nb)) != OPM_OK) return fail(s);
    S.y = y;
  } else {
    double *lu;
    if ((s = dalloc(h, &lu, (size_t)an.lu_vals)) != OPM_OK) return fail(s);
    S.lu = lu;
    double *y;
    if ((s = dalloc(h, &y, 3 * (size_t)nb)) != OPM_OK) return fail(s);
    S.y = y;
  }
  double **vecs[] = {&S.x, &S.r, &S.rh, &S.p, &S.v, &S.ph, &S.s, &S.sh, &S.t, &S.w, &h->vec_in, &h->vec_out};
  for (double **pv : vecs)
    if ((s = dalloc(h, pv, 3 * (size_t)nb)) != OPM_OK) return fail(s);
  if ((s = dalloc(h, &S.partials, 4 * (size_t)h->ntiles)) != OPM_OK) return fail(s);
  if ((s = dalloc(h, &S.st, 1)) != OPM_OK) return fail(s);
  {
    DevState init{};
    init.status = OPM_OK;
    *h->h_state = init;
    if (cudaMemcpyAsync(S.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return fail(OPM_ERR_CUDA);
  }
  h->cooperative = o.sweep_launch == OPM_SWEEP_COOPERATIVE ||
                   (o.sweep_launch == OPM_SWEEP_AUTO && S.nphases > kMaxPhaseLaunches);
  const int mps = max_phase_slices(an);
  if (h->fp32) {
    h->grid_apply = apply_grid<float>(h->device, mps);
    h->grid_factor = resident_grid(k_factor<float>, h->device, mps);
  } else {
    h->grid_apply = apply_grid<double>(h->device, mps);
    h->grid_factor = resident_grid(k_factor<double>, h->device, mps);
  }
  // free the host copies the device now holds (keep perm and the factor slots)
  std::vector<int32_t>().swap(an.a_col);
  std::vector<int32_t>().swap(an.a_src);
  std::vector<int64_t>().swap(an.a_dst);
  std::vector<int32_t>().swap(an.l_col);
  std::vector<int32_t>().swap(an.u_col);
  std::vector<int32_t>().swap(an.upd_ptr);
  std::vector<int64_t>().swap(an.upd_dst);
  std::vector<int64_t>().swap(an.upd_src);


  if (o.profile_kernels && nb > 0) {
    h->kev.assign((size_t)6 * h->chunk, nullptr);
    for (auto &e : h->kev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return fail(OPM_ERR_CUDA);
      }
  }
  if (nb > 0 && (s = build_graph(h)) != OPM_OK) return fail(s);
  s = factor_impl(h, nb > 0 ? vals : nullptr);
  if (s == OPM_ERR_ZERO_PIVOT) {
    // the handle stays usable: the row can be read and new values factored
    *out = h;
    return s;
  }
  if (s != OPM_OK) return fail(s);
  *out = h;
  return OPM_OK;
}

opm_status opm_ilu0_factor(opm_handle h, const double *vals) {
  if (!h) return OPM_ERR_ARG;
  h->last_err_row = -1;
  return factor_impl(h, vals);
}

opm_status opm_bicgstab_solve(opm_handle h, const double *b, double *x, double rtol, int32_t maxit,
                              int32_t *iters, double *relres) {
  if (!h || (h->n > 0 && (!b || !x)) || !(rtol >= 0.0)) return OPM_ERR_ARG;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (h->n == 0) return OPM_OK;
  if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  const size_t vbytes = sizeof(double) * 3 * (size_t)h->n;
  const double *db = nullptr;
  opm_status s = stage_in(h, b, &db);
  if (s != OPM_OK) return s;
  const bool x_dev = is_device_ptr(x);
  double *dx = x_dev ? x : h->vec_out;
  cudaStream_t st = h->stream;
  CK(cudaEventRecord(h->ev[0], st));
  k_setup<<<h->ntiles, 256, 0, st>>>(h->sys, db, rtol, maxit);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev[1], st));
  h->timing.launches += 1;
  if ((s = read_state(h)) != OPM_OK) return s;
  while (h->h_state->status == kRunning && h->h_state->error == 0) {
    const int k_before = h->h_state->k;
    CK(cudaGraphLaunch(h->chunk_exec, st));
    h->timing.launches += h->chunk_launches;
    if ((s = read_state(h)) != OPM_OK) return s;
    if (!h->kev.empty()) {
      // iterations of this chunk that did work
      int ran = h->chunk;
      if (h->h_state->status != kRunning || h->h_state->error != 0)
        ran = std::max(0, std::min(h->chunk, h->h_state->iters - k_before + 1));
      for (int it = 0; it < ran; ++it)
        for (int q = 0; q < 5; ++q) add_kernel_time(h, kIterKernel[q], h->kev[6 * it + q], h->kev[6 * it + q + 1]);
    }
  }
  CK(cudaEventRecord(h->ev[2], st));
  int32_t status = h->h_state->error != 0 ? h->h_state->error : h->h_state->status;
  if (status == OPM_OK || status == OPM_NOT_CONVERGED) {
    k_finish<<<h->ntiles, 1024, 0, st>>>(h->sys, db, dx);
    CK(cudaGetLastError());
    if (!x_dev) CK(cudaMemcpyAsync(x, dx, vbytes, cudaMemcpyDeviceToHost, st));
  } else if (x_dev) {
    CK(cudaMemsetAsync(x, 0, vbytes, st));
  } else {
    memset(x, 0, vbytes);
  }
  CK(cudaEventRecord(h->ev[3], st));
  if (status == OPM_OK || status == OPM_NOT_CONVERGED) h->timing.launches += 1;
  if ((s = read_state(h)) != OPM_OK) return s;
  if (h->opt.profile_kernels) {
    add_kernel_time(h, OPM_KERNEL_SETUP, h->ev[0], h->ev[1]);
    if (status == OPM_OK || status == OPM_NOT_CONVERGED) add_kernel_time(h, OPM_KERNEL_FINISH, h->ev[2], h->ev[3]);
  }
  cudaEventElapsedTime(&h->timing.setup_ms, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(&h->timing.iterate_ms, h->ev[1], h->ev[2]);
  cudaEventElapsedTime(&h->timing.finish_ms, h->ev[2], h->ev[3]);
  if (iters) *iters = h->h_state->iters;
  if (relres) *relres = (status == OPM_OK || status == OPM_NOT_CONVERGED) ? h->h_state->relres : NAN;
  return (opm_status)status;
}

opm_status opm_spmv(opm_handle h, const double *x, double *y) {
  if (!h || (h->n > 0 && (!x || !y))) return OPM_ERR_ARG;
  if (h->n == 0) return OPM_OK;
  const double *dx = nullptr;
  opm_status s = stage_in(h, x, &dx);
  if (s != OPM_OK) return s;
  const bool y_dev = is_device_ptr(y);
  double *dy = y_dev ? y : h->vec_out;
  k_gather<<<h->ntiles, 256, 0, h->stream>>>(h->sys, dx, h->sys.w);
  k_spmv_plain<<<h->ntiles, 1024, 0, h->stream>>>(h->sys, h->sys.w, dy);
  CK(cudaGetLastError());
  h->timing.launches += 2;
  if (!y_dev) CK(cudaMemcpyAsync(y, dy, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OPM_OK;
}

opm_status opm_ilu_apply(opm_handle h, const double *r, double *z) {
  if (!h || (h->n > 0 && (!r || !z))) return OPM_ERR_ARG;
  if (h->n == 0) return OPM_OK;
  if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  const double *dr = nullptr;
  opm_status s = stage_in(h, r, &dr);
  if (s != OPM_OK) return s;
  const bool z_dev = is_device_ptr(z);
  double *dz = z_dev ? z : h->vec_out;
  k_begin_factor<<<1, 1, 0, h->stream>>>(h->sys.st);
  k_gather<<<h->ntiles, 256, 0, h->stream>>>(h->sys, dr, h->sys.w);
  const int nl = launch_apply_p<kModePlain>(h, h->sys.w, h->sys.t, h->stream);
  k_scatter<<<h->ntiles, 256, 0, h->stream>>>(h->sys, h->sys.t, dz);
  CK(cudaGetLastError());
  h->timing.launches += 3 + nl;
  if (!z_dev) CK(cudaMemcpyAsync(z, dz, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  if ((s = read_state(h)) != OPM_OK) return s;
  if (h->h_state->error != 0) return (opm_status)h->h_state->error;
  return OPM_OK;
}

int32_t opm_last_error_row(opm_handle h) { return h ? h->last_err_row : t_create_err_row; }

opm_status opm_get_info(opm_handle h, opm_info *info) {
  if (!h || !info) return OPM_ERR_ARG;
  info->nb = h->n;
  info->schedule = h->an.schedule;
  info->precision = h->fp32 ? OPM_PREC_FP32_FACTORS : OPM_PREC_FP64;
  info->nsets = h->an.nsets;
  info->nnzb = h->nnzb;
  info->nnzb_lower = h->an.nnz_l;
  info->nnzb_upper = h->an.nnz_u;
  info->device_bytes = h->dev_bytes;
  info->nphases = h->sys.nphases;
  info->reserved = 0;
  return OPM_OK;
}

opm_status opm_get_permutation(opm_handle h, int32_t *perm) {
  if (!h || (!perm && h->n > 0)) return OPM_ERR_ARG;
  if (h->n > 0) memcpy(perm, h->an.perm.data(), sizeof(int32_t) * (size_t)h->n);
  return OPM_OK;
}

opm_status opm_get_factors(opm_handle h, double *lu, double *dinv) {
  if (!h) return OPM_ERR_ARG;
  if (h->n == 0) return OPM_OK;
  const Analysis &an = h->an;
  std::vector<double> v((size_t)an.lu_vals);
  if (h->fp32) {
    std::vector<float> f((size_t)an.lu_vals);
    CK(cudaMemcpyAsync(f.data(), h->sys.lu, sizeof(float) * f.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t e = 0; e < f.size(); ++e) v[e] = (double)f[e];
  } else {
    CK(cudaMemcpyAsync(v.data(), h->sys.lu, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  if (lu) {
    for (int64_t c = 0; c < h->nnzb; ++c) {
      const int64_t slot = an.a_csr_slot[c];
      const int64_t off = slot >> 6;
      const int st = (int)(slot & 63);
      for (int e = 0; e < 9; ++e) lu[9 * c + e] = v[off + (int64_t)e * st];
    }
  }
  if (dinv) {
    for (int32_t i = 0; i < h->n; ++i)
      for (int e = 0; e < 9; ++e)
        dinv[9 * (int64_t)i + e] = v[an.d_off + (int64_t)kSliceVals * (i / kWarp) + 32 * e + (i % kWarp)];
  }
  return OPM_OK;
}

opm_status opm_get_timing(opm_handle h, opm_timing *t) {
  if (!h || !t) return OPM_ERR_ARG;
  *t = h->timing;
  return OPM_OK;
}

opm_status opm_reset_timing(opm_handle h) {
  if (!h) return OPM_ERR_ARG;
  h->timing.launches = 0;
  for (int k = 0; k < OPM_KERNEL_COUNT; ++k) {
    h->timing.kernel_ms[k] = 0.0;
    h->timing.kernel_count[k] = 0;
  }
  return OPM_OK;
}

}  // extern "C"
