// Host driver and C ABI of the GB300 BSR ILU0-BiCGStab library.
//
// A handle owns one system's schedule-ordered device copy of the matrix, its
// ILU0 factors and its Krylov vectors.  Work is launched through a Runner: a
// set of systems (a handle's own set of one, or a batch of handles) with its
// work lists, its kernel-parameter block and three CUDA graphs:
//   * factor graph: clear errors -> ILU0 phases -> record errors -> results;
//   * solve graph: setup -> while (any system running) { `chunk` BiCGStab
//     iterations; loop condition } -> true residual -> results.  The loop
//     runs on the device (a conditional graph node): one graph launch per
//     solve, no host round trip between iterations;
//   * iteration graph (only with profile_kernels): `chunk` iterations with
//     event-record nodes between kernels, driven by a host loop, for
//     per-kernel device times.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "sweeps.cuh"
#include "factor.cuh"
#include "gmres.cuh"
#include "iterative.cuh"

using namespace opm;

namespace opm {
struct Runner;
}

struct opm_solver {
  Analysis an;
  opm_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int32_t n = 0, nslices = 0, ntiles = 0;
  int64_t nnzb = 0;
  bool fp32 = false;
  Sys sys{};                     // this system's descriptor (host copy)
  std::vector<void *> allocs;
  std::vector<void *> well_allocs;  // arrays of the current wells (replaced by opm_set_wells)
  double *gm_V = nullptr;           // GMRES: Krylov basis, gm_m + 1 vectors
  double *gm_part = nullptr;        // GMRES: per-tile partial sums
  int gm_m = 0;
  opm::GmState *gm_state = nullptr; // GMRES: device-side control state
  opm::GmState *gm_hstate = nullptr;  // GMRES: pinned host copy (inputs and outcome)
  cudaGraphExec_t gm_exec = nullptr;  // GMRES: the whole solve, built on first use
  double *gm_exec_V = nullptr;        // basis the graph was built for
  bool gm_exec_wells = false;         // wells the graph was built for
  int64_t dev_bytes = 0;
  double *vals_stage = nullptr;  // caller's values when given from host
  double *vec_in = nullptr, *vec_out = nullptr;  // caller-order staging
  int32_t last_err_row = -1;
  bool factors_ok = false;
  opm_timing timing{};
  cudaEvent_t ev[2] = {};
  opm::Runner *run = nullptr;    // batch of one
  bool async_pending = false;
};

struct opm_analysis_s {
  opm::Analysis an;  // the whole analysis, device lists included
};

struct opm_batch_s {
  opm::Runner *run = nullptr;
  std::vector<opm_solver *> members;
  std::vector<char> sat_out;  // members that sit the pending launch out
  bool async_pending = false;
};

namespace opm {

struct Runner {
  std::vector<opm_solver *> mem;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool fp32 = false, cooperative = false, profile = false;
  bool reuse = false;     // products after an application use Sys::uz (opm_options.product_reuse)
  int chunk = 2, nsys = 0, nphases = 0, ntiles = 0, ntiles_s = 0;
  int small_entries = 0;  // sweep phases with at most this many slices take the latency form
  int sms = 1;            // SMs of the device
  int cp_sweeps = 0;      // > 0: iterative ILU0 with this many sweeps instead of the phases
  int tri_sweeps = 0;     // > 0: Jacobi triangular solves with this many sweeps per triangle
  int nall = 0;           // slices of all systems (the iterative kernels' work list)
  bool has_wells = false; // some member has wells: products launch k_wells first (graphs built so)
  std::vector<int32_t> fwd_ptr, bwd_ptr;
  Batch B{};
  Sys *h_sys = nullptr;      // pinned staging of the descriptors
  Result *h_res = nullptr;   // pinned results
  size_t h_sys_cls = 0, h_res_cls = 0;  // their size classes in the pinned free list
  Result *d_res = nullptr;
  std::vector<void *> allocs;
  int64_t dev_bytes = 0;
  int grid_apply = 1, grid_factor = 1;
  cudaGraphExec_t solve_exec = nullptr, iter_exec = nullptr, factor_exec = nullptr;
  cudaGraphExec_t fs_exec = nullptr;  // refactor + solve in one graph (setup beside the factorisation)
  int iter_launches = 0, factor_launches = 0;
  std::vector<cudaEvent_t> kev;  // profiling events, 6 per iteration of a chunk
  cudaEvent_t ev_done = nullptr;
};

}  // namespace opm

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

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      fprintf(stderr, "opm_bsr: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      cudaGetLastError();                                                         \
      return e_ == cudaErrorMemoryAllocation ? OPM_ERR_OOM : OPM_ERR_CUDA;        \
    }                                                                             \
  } while (0)

std::mutex &pinned_mutex() {
  static std::mutex mu;
  return mu;
}

std::map<size_t, std::vector<void *>> &pinned_free_list() {
  static std::map<size_t, std::vector<void *>> fl;
  return fl;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory of handles, batches and wells comes from one memory pool per
// device, allocated and freed in stream order (cudaMallocFromPoolAsync /
// cudaFreeAsync on the owner's stream), and the pool keeps what is freed
// for the next allocation.  Unlike cudaMalloc / cudaFree, creating or
// destroying a handle then does not serialise with work running on other
// streams (a serving loop evicting and remaking instances while others
// solve).  The pool's memory stays with the process.
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
    pools[dev] = pool;
  }
  return pools[dev];
}

template <typename T>
opm_status dalloc(std::vector<void *> &allocs, int64_t &bytes_acc, cudaStream_t st, T **p, size_t count) {
  *p = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaMemPool_t pool = device_pool();
  if (!pool) return OPM_ERR_CUDA;
  cudaError_t e = cudaMallocFromPoolAsync((void **)p, bytes, pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? OPM_ERR_OOM : OPM_ERR_CUDA;
  }
  allocs.push_back(*p);
  bytes_acc += (int64_t)bytes;
  return OPM_OK;
}

// Frees allocations of dalloc in stream order on st.
void dfree(std::vector<void *> &allocs, cudaStream_t st) {
  for (void *p : allocs) cudaFreeAsync(p, st);
  allocs.clear();
  cudaGetLastError();
}

// Page-locked host buffers of batches (descriptors, results), kept in a
// process-wide free list by size class: cudaMallocHost blocks concurrency
// with other streams, so it runs only when no freed buffer of the size is
// left.
void *pinned_alloc(size_t bytes, size_t *cls) {
  static_assert(sizeof(size_t) >= 8, "64-bit sizes");
  size_t c = 256;
  while (c < bytes) c <<= 1;
  *cls = c;
  std::lock_guard<std::mutex> lock(pinned_mutex());
  auto &fl = pinned_free_list()[c];
  if (!fl.empty()) {
    void *p = fl.back();
    fl.pop_back();
    return p;
  }
  void *p = nullptr;
  if (cudaMallocHost(&p, c) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pinned_release(void *p, size_t cls) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(pinned_mutex());
  pinned_free_list()[cls].push_back(p);
}

template <typename T>
opm_status upload(std::vector<void *> &allocs, int64_t &bytes_acc, cudaStream_t st, T **p,
                  const std::vector<T> &v) {
  opm_status s = dalloc(allocs, bytes_acc, st, p, v.size());
  if (s != OPM_OK) return s;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return OPM_OK;
}

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

// Kernels inside the iteration graph are launched with programmatic stream
// serialization: the next kernel's CTAs may be scheduled while the previous
// kernel drains, and wait in griddepcontrol.wait for its completion.
template <typename... P, typename... A>
void launch_pdl(void (*kern)(P...), int grid, int block, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// Schedules with at most this many phases run one launch per phase; more
// phases run as one cooperative launch with grid barriers.
constexpr int kMaxPhaseLaunches = 1024;

// Bounds of the iterative sweeps (each sweep is a node of the captured graphs).
constexpr int kMaxCpSweeps = 4096;
constexpr int kMaxTriSweeps = 64;

int blocks8(int entries) { return std::max(1, (entries + 7) / 8); }

// Iterative ILU0: the initial guess, then cp_sweeps synchronous sweeps,
// alternating between the two factor buffers so that the last sweep writes
// the one the solver reads (sweep t of T writes buffer (T - t) & 1).
template <typename TF>
int launch_cp_factor_t(Runner &R, cudaStream_t st) {
  const int T = R.cp_sweeps, g = blocks8(R.nall);
  launch_pdl(k_cp_init<TF>, g, 256, st, R.B, 0, T & 1);
  launch_pdl(k_cp_init<TF>, g, 256, st, R.B, 1, T & 1);
  for (int t = 1; t <= T; ++t) launch_pdl(k_cp_sweep<TF>, g, 256, st, R.B, (T - t) & 1);
  return T + 2;
}

template <typename TF>
int launch_factor_t(Runner &R, cudaStream_t st) {
  if (R.cp_sweeps > 0) return launch_cp_factor_t<TF>(R, st);
  if (R.cooperative) {
    launch_coop(k_factor<TF>, R.grid_factor, st, R.B);
    return 1;
  }
  // A small phase is bound by the FP64 rate of the SMs it occupies (a few
  // warps per row, dozens of FMAs per block): two warps per CTA spread it
  // over up to all SMs instead of one in eight.
  constexpr bool kFp32 = sizeof(TF) == 4;
  int n = 0;
  for (int c = 0; c < R.nphases; ++c) {
    const int cnt = R.fwd_ptr[c + 1] - R.fwd_ptr[c];
    if (cnt == 0) continue;
    if (cnt <= R.small_entries) launch_pdl(k_factor_phase<TF, kFp32, 1>, (cnt + 1) / 2, 64, st, R.B, c);
    else launch_pdl(k_factor_phase<TF, true, 4, kFp32>, blocks8(cnt), 256, st, R.B, c);
    ++n;
  }
  return n;
}

// Slabs a small-phase sweep loads ahead of its wait: 8 covers nearly every
// row of the small colours (high-degree rows) and fits the 255-register
// budget without spills for FP64 blocks.
template <typename TF>
constexpr int sweep_preload() {
  return 8;
}

// One phase of a sweep: phases of at most R.small_entries slices take the
// latency form (two warps per CTA, constant data loaded before the wait),
// larger ones the throughput form.
template <typename TF, int MODE, bool FWD>
void launch_sweep_phase(Runner &R, cudaStream_t st, int c, int cnt) {
  constexpr int P = sweep_preload<TF>();
  if (cnt <= R.small_entries) {
    if (FWD) launch_pdl(k_fwd_phase<TF, MODE, P>, (cnt + 1) / 2, 64, st, R.B, c);
    else launch_pdl(k_bwd_phase<TF, MODE, P>, (cnt + 1) / 2, 64, st, R.B, c);
  } else {
    if (FWD) launch_pdl(k_fwd_phase<TF, MODE, 0>, blocks8(cnt), 256, st, R.B, c);
    else launch_pdl(k_bwd_phase<TF, MODE, 0>, blocks8(cnt), 256, st, R.B, c);
  }
}

// Jacobi triangular solves: the right-hand side (MODE P / S), tri_sweeps
// forward sweeps, tri_sweeps backward sweeps.
template <typename TF, int MODE>
int launch_jacobi_apply_t(Runner &R, cudaStream_t st) {
  const int T = R.tri_sweeps, g = blocks8(R.nall);
  int n = 2 * T;
  if constexpr (MODE != kModePlain) {
    launch_pdl(k_jac_rhs<MODE>, R.ntiles, 256, st, R.B);
    ++n;
  }
  for (int t = 1; t <= T; ++t) launch_pdl(k_jac_fwd<TF, MODE>, g, 256, st, R.B, t, T);
  for (int t = 1; t <= T; ++t) launch_pdl(k_jac_bwd<TF, MODE>, g, 256, st, R.B, t, T);
  return n;
}

template <typename TF, int MODE>
int launch_apply_t(Runner &R, cudaStream_t st) {
  if (R.tri_sweeps > 0) return launch_jacobi_apply_t<TF, MODE>(R, st);
  if (R.cooperative) {
    launch_coop(k_apply<TF, MODE>, R.grid_apply, st, R.B);
    return 1;
  }
  int n = 0;
  for (int c = 0; c < R.nphases; ++c) {
    const int cnt = R.fwd_ptr[c + 1] - R.fwd_ptr[c];
    if (cnt == 0) continue;
    if (c == 0) launch_pdl(k_fwd_first<TF, MODE>, blocks8(cnt), 256, st, R.B);  // no L blocks in phase 0
    else launch_sweep_phase<TF, MODE, true>(R, st, c, cnt);
    ++n;
  }
  for (int c = R.nphases - 1; c >= 0; --c) {
    const int cnt = R.bwd_ptr[c + 1] - R.bwd_ptr[c];
    if (cnt == 0) continue;
    launch_sweep_phase<TF, MODE, false>(R, st, c, cnt);
    ++n;
  }
  return n;
}

template <int MODE>
int launch_apply(Runner &R, cudaStream_t st) {
  return R.fp32 ? launch_apply_t<float, MODE>(R, st) : launch_apply_t<double, MODE>(R, st);
}

int launch_factor_seq(Runner &R, cudaStream_t st) {
  const int sb = std::max(1, (R.nsys + 255) / 256);
  k_begin_factor<<<sb, 256, 0, st>>>(R.B);
  const int n = R.fp32 ? launch_factor_t<float>(R, st) : launch_factor_t<double>(R, st);
  k_end_factor<<<sb, 256, 0, st>>>(R.B);
  return n + 2;
}

// One BiCGStab iteration.  With ev (6 events), the kernel groups are
// bracketed by event-record nodes (external records, so that they become
// real graph nodes) for per-kernel timing.
int launch_iteration(Runner &R, cudaStream_t st, cudaEvent_t *ev) {
  auto mark = [&](int q) {
    if (ev) cudaEventRecordWithFlags(ev[q], st, cudaEventRecordExternal);
  };
  int n = 3;
  mark(0);
  n += launch_apply<kModeP>(R, st);
  mark(1);
  if (R.has_wells) {
    launch_pdl(k_wells, R.nsys, 256, st, R.B, 0);
    ++n;
  }
  if (R.reuse) launch_pdl(k_spmv_v<true>, R.ntiles_s, 256, st, R.B);
  else launch_pdl(k_spmv_v<false>, R.ntiles_s, 256, st, R.B);
  mark(2);
  n += launch_apply<kModeS>(R, st);
  mark(3);
  if (R.has_wells) {
    launch_pdl(k_wells, R.nsys, 256, st, R.B, 1);
    ++n;
  }
  if (R.reuse && R.ntiles_s > 6 * R.sms) launch_pdl(k_spmv_t<true, true>, R.ntiles_s, 256, st, R.B);
  else if (R.reuse) launch_pdl(k_spmv_t<true, false>, R.ntiles_s, 256, st, R.B);
  else launch_pdl(k_spmv_t<false>, R.ntiles_s, 256, st, R.B);
  mark(4);
  launch_pdl(k_update, R.ntiles, 256, st, R.B);
  mark(5);
  return n;
}

const int kIterKernel[5] = {OPM_KERNEL_APPLY, OPM_KERNEL_SPMV, OPM_KERNEL_APPLY, OPM_KERNEL_SPMV,
                            OPM_KERNEL_UPDATE};

void add_kernel_time(opm_timing &t, int kind, cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
    t.kernel_ms[kind] += ms;
    t.kernel_count[kind] += 1;
  } else {
    cudaGetLastError();
  }
}

int results_blocks(const Runner &R) { return std::max(1, (R.nsys + 127) / 128); }

template <typename K>
int resident_grid(K kernel, int device, int items) {
  int sms = 1, occ = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kSweepThreads, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int warps = kSweepThreads / 32;
  return std::max(1, std::min(sms * occ, (items + warps - 1) / warps));
}

template <typename TF>
void cooperative_grids(Runner &R, int max_entries) {
  int g = resident_grid(k_apply<TF, kModeP>, R.device, max_entries);
  g = std::min(g, resident_grid(k_apply<TF, kModeS>, R.device, max_entries));
  R.grid_apply = std::min(g, resident_grid(k_apply<TF, kModePlain>, R.device, max_entries));
  R.grid_factor = resident_grid(k_factor<TF>, R.device, max_entries);
}

opm_status add_kernel_node(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep, size_t ndep,
                           void *func, int grid, int block, void **args) {
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  CK(cudaGraphAddKernelNode(node, g, dep, ndep, &kp));
  return OPM_OK;
}

// Adds, after node dep of graph g: the device-side iteration loop (a
// conditional while node whose body holds `chunk` iterations and the loop
// condition), the wells' final term, the true residual and the results.
opm_status add_solve_loop(Runner &R, cudaGraph_t g, cudaGraphNode_t dep, cudaStream_t cap) {
  opm_status s = OPM_OK;
  void *argsB[] = {&R.B};
  cudaGraphNode_t n_while, n_finish, n_res;
  cudaGraphConditionalHandle ch;
  if (cudaGraphConditionalHandleCreate(&ch, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return OPM_ERR_CUDA;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = ch;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(&n_while, g, &dep, nullptr, 1, &cp) != cudaSuccess) return OPM_ERR_CUDA;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return OPM_ERR_CUDA;
  R.iter_launches = 0;
  for (int it = 0; it < R.chunk; ++it) R.iter_launches = launch_iteration(R, cap, nullptr);
  k_loop_cond<<<1, 256, 0, cap>>>(R.B, ch);
  if (cudaStreamEndCapture(cap, &body) != cudaSuccess) return OPM_ERR_CUDA;
  cudaGraphNode_t n_pre = n_while;
  int which_x = 2;
  void *argsW[] = {&R.B, &which_x};
  if (R.has_wells && (s = add_kernel_node(g, &n_pre, &n_while, 1, (void *)k_wells, R.nsys, 256, argsW)) != OPM_OK)
    return s;
  if ((s = add_kernel_node(g, &n_finish, &n_pre, 1, (void *)k_finish, R.ntiles_s, 256, argsB)) != OPM_OK) return s;
  void *argsR[] = {&R.B, &R.d_res};
  return add_kernel_node(g, &n_res, &n_finish, 1, (void *)k_results, results_blocks(R), 128, argsR);
}

opm_status build_graphs(Runner &R) {
  cudaStream_t cap;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  opm_status s = OPM_OK;
  cudaGraph_t g = nullptr, fg = nullptr;
  // ---- factor graph
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    s = OPM_ERR_CUDA;
  } else {
    R.factor_launches = launch_factor_seq(R, cap) + 1;
    k_results<<<results_blocks(R), 128, 0, cap>>>(R.B, R.d_res);
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess || cudaGraphInstantiate(&R.factor_exec, g, 0) != cudaSuccess)
      s = OPM_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  g = nullptr;
  void *argsB[] = {&R.B};
  // ---- solve graph: setup, then the device-side iteration loop
  if (s == OPM_OK) {
    cudaGraphNode_t n_setup;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) s = OPM_ERR_CUDA;
    if (s == OPM_OK) s = add_kernel_node(g, &n_setup, nullptr, 0, (void *)k_setup<true>, R.ntiles, 256, argsB);
    if (s == OPM_OK) s = add_solve_loop(R, g, n_setup, cap);
    if (s == OPM_OK && cudaGraphInstantiate(&R.solve_exec, g, 0) != cudaSuccess) s = OPM_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  g = nullptr;
  // ---- refactor + solve graph: the factorisation and the setup's vector
  // work run as independent branches (the setup needs only b), joined by
  // k_start, which applies the factorisation's outcome to the solve state.
  // Not with cooperative launches, which must own the whole device.
  if (s == OPM_OK && !R.cooperative) {
    cudaGraphNode_t n_fac, n_setup, n_start;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      s = OPM_ERR_CUDA;
    } else {
      launch_factor_seq(R, cap);
      if (cudaStreamEndCapture(cap, &fg) != cudaSuccess) s = OPM_ERR_CUDA;
    }
    if (s == OPM_OK && cudaGraphCreate(&g, 0) != cudaSuccess) s = OPM_ERR_CUDA;
    if (s == OPM_OK && cudaGraphAddChildGraphNode(&n_fac, g, nullptr, 0, fg) != cudaSuccess) s = OPM_ERR_CUDA;
    if (s == OPM_OK) s = add_kernel_node(g, &n_setup, nullptr, 0, (void *)k_setup<false>, R.ntiles, 256, argsB);
    cudaGraphNode_t deps[2] = {n_fac, n_setup};
    if (s == OPM_OK) s = add_kernel_node(g, &n_start, deps, 2, (void *)k_start, results_blocks(R), 128, argsB);
    if (s == OPM_OK) s = add_solve_loop(R, g, n_start, cap);
    if (s == OPM_OK && cudaGraphInstantiate(&R.fs_exec, g, 0) != cudaSuccess) s = OPM_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  if (fg) cudaGraphDestroy(fg);
  g = nullptr;
  // ---- profiled iteration graph
  if (s == OPM_OK && R.profile) {
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      s = OPM_ERR_CUDA;
    } else {
      for (int it = 0; it < R.chunk; ++it) launch_iteration(R, cap, &R.kev[6 * it]);
      k_results<<<results_blocks(R), 128, 0, cap>>>(R.B, R.d_res);
      if (cudaStreamEndCapture(cap, &g) != cudaSuccess || cudaGraphInstantiate(&R.iter_exec, g, 0) != cudaSuccess)
        s = OPM_ERR_CUDA;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (s != OPM_OK) {
    fprintf(stderr, "opm_bsr: graph construction failed: %s\n", cudaGetErrorString(cudaGetLastError()));
    cudaGetLastError();
  }
  return s;
}

void runner_destroy(Runner *R) {
  if (!R) return;
  cudaStreamSynchronize(R->stream);
  if (R->solve_exec) cudaGraphExecDestroy(R->solve_exec);
  if (R->iter_exec) cudaGraphExecDestroy(R->iter_exec);
  if (R->factor_exec) cudaGraphExecDestroy(R->factor_exec);
  if (R->fs_exec) cudaGraphExecDestroy(R->fs_exec);
  dfree(R->allocs, R->stream);
  pinned_release(R->h_sys, R->h_sys_cls);
  pinned_release(R->h_res, R->h_res_cls);
  for (auto &e : R->kev)
    if (e) cudaEventDestroy(e);
  if (R->ev_done) cudaEventDestroy(R->ev_done);
  delete R;
}

// Work lists and graphs for a set of analysed, allocated systems.
// Whether the BiCGStab products after an application take their upper sums
// from the backward sweep (Sys::uz): FP64 factors (an FP32 U is not A's to
// FP64 accuracy) and exact triangular solves (a Jacobi-swept p^ does not
// satisfy LU p^ = p), unless the options turn it off.
bool product_reuse_applies(const opm_options &o, bool fp32) {
  return !fp32 && o.tri_sweeps == 0 && o.product_reuse == 0;
}

uint64_t spin_ns(const opm_options &o) {
  return (uint64_t)(o.spin_limit_us > 0 ? o.spin_limit_us : 2000000) * 1000ull;
}

int chunk_of(const opm_options &o) { return o.chunk > 0 ? o.chunk : 2; }

opm_status runner_create(const std::vector<opm_solver *> &mem, cudaStream_t stream, const opm_options &o,
                         Runner **out) {
  const int chunk = chunk_of(o), sweep_launch = o.sweep_launch, skip_cta = o.debug_skip_item;
  const bool profile = o.profile_kernels != 0;
  *out = nullptr;
  Runner *R = new (std::nothrow) Runner();
  if (!R) return OPM_ERR_OOM;
  auto fail = [&](opm_status s) {
    runner_destroy(R);
    return s;
  };
  R->mem = mem;
  R->stream = stream;
  R->nsys = (int)mem.size();
  R->fp32 = mem[0]->fp32;
  R->chunk = chunk;
  R->profile = profile;
  if (cudaGetDevice(&R->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_CUDA);
  }
  int sms = 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, R->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_CUDA);
  }
  R->small_entries = o.small_phase_slices > 0 ? o.small_phase_slices : o.small_phase_slices < 0 ? 0 : 10 * sms;
  R->sms = sms;
  R->cp_sweeps = o.cp_sweeps;
  R->tri_sweeps = o.tri_sweeps;
  R->reuse = product_reuse_applies(o, R->fp32);
  // second buffers of the iterative sweeps, kept by the members
  for (auto *h : mem) {
    opm_status sa = OPM_OK;
    const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
    if (R->cp_sweeps > 0 && !h->sys.lu2) {
      uint8_t *p = nullptr;
      sa = dalloc(h->allocs, h->dev_bytes, stream, &p, esz * (size_t)h->an.lu_vals);
      h->sys.lu2 = p;
    }
    if (sa == OPM_OK && R->tri_sweeps > 0 && !h->sys.y2) {
      uint8_t *p = nullptr;
      sa = dalloc(h->allocs, h->dev_bytes, stream, &p, esz * 3 * (size_t)h->n);
      h->sys.y2 = p;
      if (sa == OPM_OK) sa = dalloc(h->allocs, h->dev_bytes, stream, &h->sys.z2, 3 * (size_t)h->n);
    }
    if (sa != OPM_OK) return fail(sa);
  }
  for (auto *h : mem) R->has_wells = R->has_wells || h->sys.nwells > 0;
  int maxp = 0;
  for (auto *h : mem) maxp = std::max(maxp, (int)h->an.phase_ptr.size() - 1);
  R->nphases = maxp;
  // ---- sweep work lists: forward entries of every phase, then backward ones
  std::vector<int4> ent;
  R->fwd_ptr.assign(1, 0);
  int max_entries = 1;
  for (int c = 0; c < maxp; ++c) {
    for (int s = 0; s < R->nsys; ++s) {
      const auto &pp = mem[s]->an.phase_ptr;
      const int np = (int)pp.size() - 1;
      if (c >= np) continue;
      const int r0 = pp[c], r1 = pp[c + 1];
      for (int sl = r0 >> 5; sl <= (r1 - 1) >> 5; ++sl) ent.push_back(make_int4(s, sl, r0, r1));
    }
    R->fwd_ptr.push_back((int)ent.size());
    max_entries = std::max(max_entries, R->fwd_ptr[c + 1] - R->fwd_ptr[c]);
  }
  // backward entries: per slice, the span of the phase's rows that have U
  // blocks (the others finish in the forward sweep)
  R->bwd_ptr.assign(1, (int)ent.size());
  for (int c = 0; c < maxp; ++c) {
    for (int s = 0; s < R->nsys; ++s) {
      const auto &pp = mem[s]->an.phase_ptr;
      const auto &mask = mem[s]->an.sl_mask;
      const int np = (int)pp.size() - 1;
      if (c >= np) continue;
      const int r0 = pp[c], r1 = pp[c + 1];
      for (int sl = r0 >> 5; sl <= (r1 - 1) >> 5; ++sl) {
        int lo = -1, hi = -1;
        for (int i = std::max(r0, sl * 32); i < std::min(r1, sl * 32 + 32); ++i)
          if (!((mask[2 * sl] >> (i & 31)) & 1u)) {
            if (lo < 0) lo = i;
            hi = i + 1;
          }
        if (lo >= 0) ent.push_back(make_int4(s, sl, lo, hi));
      }
    }
    R->bwd_ptr.push_back((int)ent.size());
  }
  std::vector<int4> all_ent;
  for (int s = 0; s < R->nsys; ++s)
    for (int sl = 0; sl < mem[s]->nslices; ++sl) all_ent.push_back(make_int4(s, sl, 0, mem[s]->n));
  R->nall = (int)all_ent.size();
  std::vector<int2> tiles, tiles_s;
  std::vector<int32_t> work_s;
  for (int s = 0; s < R->nsys; ++s) {
    for (int t = 0; t < mem[s]->sys.ntiles; ++t) tiles.push_back(make_int2(s, t));
    for (int t = 0; t < mem[s]->sys.ntiles_s; ++t) {
      tiles_s.push_back(make_int2(s, t));
      const auto &st = mem[s]->an.sp_tile;
      work_s.push_back(t < (int)st.size() ? st[t] : 0);
    }
  }
  // With the product reuse a tile's work ranges from no block (rows whose
  // product is p_i) to whole rows: the 256-row tiles of the products go
  // longest first, so the heavy ones start in the first wave and the light
  // ones fill the last.  Only the launch order changes: the reductions sum
  // per tile index, in a fixed order.
  if (R->reuse) {
    std::vector<int> ord(tiles_s.size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work_s[a] > work_s[b]; });
    std::vector<int2> sorted(tiles_s.size());
    for (size_t q = 0; q < ord.size(); ++q) sorted[q] = tiles_s[ord[q]];
    tiles_s.swap(sorted);
  }
  R->ntiles = (int)tiles.size();
  R->ntiles_s = (int)tiles_s.size();
  R->cooperative =
      sweep_launch == OPM_SWEEP_COOPERATIVE || (sweep_launch == OPM_SWEEP_AUTO && maxp > kMaxPhaseLaunches);
  // ---- device copies
  opm_status s;
  int4 *d_ent, *d_all;
  int32_t *d_fwd, *d_bwd;
  int2 *d_tiles, *d_tiles_s;
  uint32_t *d_bar;
  Sys *d_sys;
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_ent, ent)) != OPM_OK) return fail(s);
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_all, all_ent)) != OPM_OK) return fail(s);
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_fwd, R->fwd_ptr)) != OPM_OK) return fail(s);
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_bwd, R->bwd_ptr)) != OPM_OK) return fail(s);
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_tiles, tiles)) != OPM_OK) return fail(s);
  if ((s = upload(R->allocs, R->dev_bytes, stream, &d_tiles_s, tiles_s)) != OPM_OK) return fail(s);
  if ((s = dalloc(R->allocs, R->dev_bytes, stream, &d_bar, 64)) != OPM_OK) return fail(s);
  if ((s = dalloc(R->allocs, R->dev_bytes, stream, &d_sys, (size_t)R->nsys)) != OPM_OK) return fail(s);
  if ((s = dalloc(R->allocs, R->dev_bytes, stream, &R->d_res, (size_t)R->nsys)) != OPM_OK) return fail(s);
  if (cudaMemsetAsync(d_bar, 0, 64 * sizeof(uint32_t), stream) != cudaSuccess) return fail(OPM_ERR_CUDA);
  R->h_sys = static_cast<Sys *>(pinned_alloc(sizeof(Sys) * R->nsys, &R->h_sys_cls));
  R->h_res = static_cast<Result *>(pinned_alloc(sizeof(Result) * R->nsys, &R->h_res_cls));
  if (!R->h_sys || !R->h_res) {
    cudaGetLastError();
    return fail(OPM_ERR_OOM);
  }
  if (cudaEventCreateWithFlags(&R->ev_done, cudaEventDisableTiming) != cudaSuccess) return fail(OPM_ERR_CUDA);
  R->B.sys = d_sys;
  R->B.ent = d_ent;
  R->B.fwd_ptr = d_fwd;
  R->B.bwd_ptr = d_bwd;
  R->B.tiles = d_tiles;
  R->B.tiles_s = d_tiles_s;
  R->B.all_ent = d_all;
  R->B.nall = R->nall;
  R->B.ntiles_s = R->ntiles_s;
  R->B.bar = d_bar;
  R->B.nsys = R->nsys;
  R->B.nphases = maxp;
  R->B.ntiles = R->ntiles;
  R->B.skip_cta = skip_cta;
  R->B.spin_limit_ns = spin_ns(o);
  if (R->fp32) cooperative_grids<float>(*R, max_entries);
  else cooperative_grids<double>(*R, max_entries);
  if (profile) {
    R->kev.assign((size_t)6 * chunk, nullptr);
    for (auto &e : R->kev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return fail(OPM_ERR_CUDA);
      }
  }
  if ((s = build_graphs(*R)) != OPM_OK) return fail(s);
  if (cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_CUDA);
  }
  *out = R;
  return OPM_OK;
}

// Copy the members' descriptors (with their per-call fields) to the device.
// Graphs for the members' current wells: the products launch k_wells only
// when some member has wells, so a change of that rebuilds the graphs.
opm_status runner_sync_wells(Runner &R) {
  bool any = false;
  for (auto *h : R.mem) any = any || h->sys.nwells > 0;
  if (any == R.has_wells) return OPM_OK;
  CK(cudaStreamSynchronize(R.stream));
  if (R.solve_exec) cudaGraphExecDestroy(R.solve_exec);
  if (R.iter_exec) cudaGraphExecDestroy(R.iter_exec);
  if (R.factor_exec) cudaGraphExecDestroy(R.factor_exec);
  if (R.fs_exec) cudaGraphExecDestroy(R.fs_exec);
  R.solve_exec = R.iter_exec = R.factor_exec = R.fs_exec = nullptr;
  R.has_wells = any;
  return build_graphs(R);
}

opm_status runner_push(Runner &R) {
  opm_status ws = runner_sync_wells(R);
  if (ws != OPM_OK) return ws;
  for (int s = 0; s < R.nsys; ++s) {
    R.h_sys[s] = R.mem[s]->sys;
    if (!R.reuse) R.h_sys[s].uz = nullptr;
  }
  CK(cudaMemcpyAsync((void *)R.B.sys, R.h_sys, sizeof(Sys) * R.nsys, cudaMemcpyHostToDevice, R.stream));
  return OPM_OK;
}

opm_status runner_pull_results(Runner &R) {
  CK(cudaMemcpyAsync(R.h_res, R.d_res, sizeof(Result) * R.nsys, cudaMemcpyDeviceToHost, R.stream));
  return OPM_OK;
}

// Enqueue (no host wait): optional factorisation, then an optional solve.
opm_status runner_enqueue(Runner &R, bool factor, bool solve) {
  opm_status s = runner_push(R);
  if (s != OPM_OK) return s;
  if (factor && solve && R.fs_exec) {
    CK(cudaGraphLaunch(R.fs_exec, R.stream));
  } else {
    if (factor) CK(cudaGraphLaunch(R.factor_exec, R.stream));
    if (solve) CK(cudaGraphLaunch(R.solve_exec, R.stream));
  }
  if ((s = runner_pull_results(R)) != OPM_OK) return s;
  CK(cudaEventRecord(R.ev_done, R.stream));
  return OPM_OK;
}

opm_status runner_wait(Runner &R) {
  CK(cudaEventSynchronize(R.ev_done));
  return OPM_OK;
}

// Kernel launches of one solve-graph execution, for the launch counter.
int64_t solve_graph_launches(const Runner &R) {
  int maxit = 1;
  for (int s = 0; s < R.nsys; ++s) maxit = std::max(maxit, R.h_res[s].iters);
  const int64_t bodies = (maxit + R.chunk - 1) / R.chunk;
  return 3 + (R.has_wells ? 1 : 0) + bodies * ((int64_t)R.iter_launches * R.chunk + 1);
}

// Host-driven solve with per-kernel events (profiling).
opm_status runner_solve_profiled(Runner &R, opm_timing &t) {
  opm_status s = runner_push(R);
  if (s != OPM_OK) return s;
  cudaEvent_t e0 = R.kev[0], e1 = R.kev[1];
  CK(cudaEventRecord(e0, R.stream));
  k_setup<true><<<R.ntiles, 256, 0, R.stream>>>(R.B);
  CK(cudaEventRecord(e1, R.stream));
  CK(cudaStreamSynchronize(R.stream));
  add_kernel_time(t, OPM_KERNEL_SETUP, e0, e1);
  t.launches += 1;
  std::vector<int> k_before(R.nsys, 0);
  for (;;) {
    CK(cudaGraphLaunch(R.iter_exec, R.stream));
    t.launches += (int64_t)R.iter_launches * R.chunk + 1;
    if ((s = runner_pull_results(R)) != OPM_OK) return s;
    CK(cudaStreamSynchronize(R.stream));
    // iterations of this chunk that did work: up to the last system's finish
    int ran = 0;
    bool any = false;
    for (int q = 0; q < R.nsys; ++q) {
      if (R.h_res[q].status == kRunning) {
        any = true;
        ran = R.chunk;
      } else {
        ran = std::max(ran, std::min(R.chunk, R.h_res[q].iters - k_before[q]));
      }
    }
    for (int it = 0; it < ran; ++it)
      for (int q = 0; q < 5; ++q) add_kernel_time(t, kIterKernel[q], R.kev[6 * it + q], R.kev[6 * it + q + 1]);
    for (int q = 0; q < R.nsys; ++q) k_before[q] = R.h_res[q].iters;
    if (!any) break;
  }
  CK(cudaEventRecord(e0, R.stream));
  if (R.has_wells) k_wells<<<R.nsys, 256, 0, R.stream>>>(R.B, 2);
  k_finish<<<R.ntiles_s, 256, 0, R.stream>>>(R.B);
  CK(cudaEventRecord(e1, R.stream));
  k_results<<<results_blocks(R), 128, 0, R.stream>>>(R.B, R.d_res);
  t.launches += 2;
  if ((s = runner_pull_results(R)) != OPM_OK) return s;
  CK(cudaStreamSynchronize(R.stream));
  add_kernel_time(t, OPM_KERNEL_FINISH, e0, e1);
  return OPM_OK;
}

// ---------------------------------------------------------------- handles

opm_status staged_vals(opm_solver *h, const double *vals, const double **dev) {
  *dev = nullptr;
  if (!vals) return OPM_OK;
  if (is_device_ptr(vals)) {
    *dev = vals;
    return OPM_OK;
  }
  if (!h->vals_stage) {
    opm_status s = dalloc(h->allocs, h->dev_bytes, h->stream, &h->vals_stage, 9 * (size_t)h->nnzb);
    if (s != OPM_OK) return s;
  }
  CK(cudaMemcpyAsync(h->vals_stage, vals, sizeof(double) * 9 * (size_t)h->nnzb, cudaMemcpyHostToDevice,
                     h->stream));
  *dev = h->vals_stage;
  return OPM_OK;
}

opm_status staged_vec(opm_solver *h, const double *src, const double **dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return OPM_OK;
  }
  CK(cudaMemcpyAsync(h->vec_in, src, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
  *dev = h->vec_in;
  return OPM_OK;
}

opm_status factor_impl(opm_solver *h, const double *vals) {
  h->factors_ok = false;
  h->last_err_row = -1;
  if (h->n == 0) {
    h->factors_ok = true;
    return OPM_OK;
  }
  const double *dv = nullptr;
  opm_status s = staged_vals(h, vals, &dv);
  if (s != OPM_OK) return s;
  h->sys.vals_in = dv;
  Runner &R = *h->run;
  CK(cudaEventRecord(h->ev[0], h->stream));
  s = runner_enqueue(R, true, false);
  h->sys.vals_in = nullptr;
  if (s != OPM_OK) return s;
  CK(cudaEventRecord(h->ev[1], h->stream));
  if ((s = runner_wait(R)) != OPM_OK) return s;
  CK(cudaEventSynchronize(h->ev[1]));
  cudaEventElapsedTime(&h->timing.factor_ms, h->ev[0], h->ev[1]);
  h->timing.launches += R.factor_launches;
  if (h->opt.profile_kernels) add_kernel_time(h->timing, OPM_KERNEL_FACTOR, h->ev[0], h->ev[1]);
  const Result &r = R.h_res[0];
  if (r.status < 0) {
    const int32_t row = r.err_row;
    h->last_err_row = (row >= 0 && row < h->n) ? h->an.perm[row] : -1;
    return (opm_status)r.status;
  }
  h->factors_ok = true;
  return OPM_OK;
}

opm_status alloc_system(opm_solver *h, const Analysis &an) {
  Sys &S = h->sys;
  const int32_t nb = h->n;
  std::vector<void *> &A = h->allocs;
  int64_t &bytes = h->dev_bytes;
  cudaStream_t st = h->stream;
  S.n = nb;
  S.nslices = h->nslices;
  S.ntiles = h->ntiles;
  S.ntiles_s = std::max(1, (nb + kSpmvRows - 1) / kSpmvRows);
  S.nphases = (int32_t)an.phase_ptr.size() - 1;
  S.u_off = 9 * an.nnz_l;
  S.d_off = an.d_off;
  opm_status s;
  int32_t *p_perm, *p_arp, *p_acol, *p_asrc, *p_lrp, *p_lcol, *p_urp, *p_ucol, *p_upd;
  int64_t *p_adst, *p_ud, *p_us;
#define UP(ptr, vec) \
  if ((s = upload(A, bytes, st, &ptr, vec)) != OPM_OK) return s
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
  uint32_t *p_mask, *p_fz, *p_spm;
  int64_t *p_aux;
  int32_t *p_spl;
  UP(p_mask, an.sl_mask);
  UP(p_fz, an.fz_mask);
  UP(p_aux, an.a_aux);
  UP(p_spm, an.sp_mask);
  UP(p_spl, an.sp_len);
#undef UP
  S.sp_mask = reinterpret_cast<const uint2 *>(p_spm);
  S.sp_len = p_spl;
  S.fz_mask = p_fz;
  S.a_aux = p_aux;
  S.sl_mask = reinterpret_cast<const uint2 *>(p_mask);
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
  if ((s = dalloc(A, bytes, st, &S.a_val, 9 * (size_t)h->nnzb)) != OPM_OK) return s;
  if (h->fp32) {
    float *lu, *y;
    if ((s = dalloc(A, bytes, st, &lu, (size_t)an.lu_vals)) != OPM_OK) return s;
    if ((s = dalloc(A, bytes, st, &y, 3 * (size_t)nb)) != OPM_OK) return s;
    S.lu = lu;
    S.y = y;
  } else {
    double *lu, *y;
    if ((s = dalloc(A, bytes, st, &lu, (size_t)an.lu_vals)) != OPM_OK) return s;
    if ((s = dalloc(A, bytes, st, &y, 3 * (size_t)nb)) != OPM_OK) return s;
    S.lu = lu;
    S.y = y;
  }
  double **vecs[] = {&S.x, &S.r, &S.rh, &S.p, &S.v, &S.ph, &S.s, &S.sh, &S.t, &S.w, &h->vec_in, &h->vec_out};
  for (double **pv : vecs)
    if ((s = dalloc(A, bytes, st, pv, 3 * (size_t)nb)) != OPM_OK) return s;
  // the backward sweep's upper sums for the products (FP64 factors only)
  S.uz = nullptr;
  if (!h->fp32 && (s = dalloc(A, bytes, st, &S.uz, 3 * (size_t)nb)) != OPM_OK) return s;
  if ((s = dalloc(A, bytes, st, &S.partials, 4 * (size_t)S.ntiles_s)) != OPM_OK) return s;
  const size_t ngroups = ((size_t)S.ntiles_s + 31) / 32;
  if ((s = dalloc(A, bytes, st, &S.grp_partials, 4 * ngroups)) != OPM_OK) return s;
  if ((s = dalloc(A, bytes, st, &S.grp_count, ngroups)) != OPM_OK) return s;
  CK(cudaMemsetAsync(S.grp_count, 0, sizeof(uint32_t) * ngroups, st));
  if ((s = dalloc(A, bytes, st, &S.st, 1)) != OPM_OK) return s;
  DevState init{};
  init.status = OPM_OK;
  CK(cudaMemcpyAsync(S.st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return OPM_OK;
}

// Frees the lists only the device needs from a handle's own analysis once
// they are uploaded (perm, phases, masks and the factor slots stay).
void drop_device_lists(Analysis &an) {
  std::vector<int32_t>().swap(an.a_col);
  std::vector<int32_t>().swap(an.a_src);
  std::vector<int64_t>().swap(an.a_dst);
  std::vector<int32_t>().swap(an.l_col);
  std::vector<int32_t>().swap(an.u_col);
  std::vector<int32_t>().swap(an.upd_ptr);
  std::vector<int64_t>().swap(an.upd_dst);
  std::vector<int64_t>().swap(an.upd_src);
  std::vector<int64_t>().swap(an.a_aux);
  std::vector<uint32_t>().swap(an.fz_mask);
  std::vector<uint32_t>().swap(an.sp_mask);
  std::vector<int32_t>().swap(an.sp_len);
}

// The host part of an analysis a handle keeps (everything but the lists
// drop_device_lists frees), copied from a kept analysis.
void copy_host_part(Analysis &dst, const Analysis &src) {
  dst.n = src.n;
  dst.nnzb = src.nnzb;
  dst.nnz_l = src.nnz_l;
  dst.nnz_u = src.nnz_u;
  dst.nnzb_kept = src.nnzb_kept;
  dst.schedule = src.schedule;
  dst.nsets = src.nsets;
  dst.perm = src.perm;
  dst.iperm = src.iperm;
  dst.a_rowptr = src.a_rowptr;
  dst.l_rowptr = src.l_rowptr;
  dst.u_rowptr = src.u_rowptr;
  dst.a_csr_slot = src.a_csr_slot;
  dst.nupd = src.nupd;
  dst.phase_ptr = src.phase_ptr;
  dst.sl_mask = src.sl_mask;
  dst.d_off = src.d_off;
  dst.lu_vals = src.lu_vals;
  dst.max_row_len = src.max_row_len;
  dst.nnzb_product = src.nnzb_product;
  dst.rows_identity = src.rows_identity;
  dst.rows_reuse = src.rows_reuse;
  dst.sp_tile = src.sp_tile;
}

opm_status check_options(const opm_options &o) {
  if (o.schedule < OPM_SCHED_AUTO || o.schedule > OPM_SCHED_COLOUR_KEMPE) return OPM_ERR_ARG;
  if (o.precision != OPM_PREC_FP64 && o.precision != OPM_PREC_FP32_FACTORS) return OPM_ERR_ARG;
  if (o.chunk < 0 || o.spin_limit_us < 0) return OPM_ERR_ARG;
  if (o.sweep_launch < OPM_SWEEP_AUTO || o.sweep_launch > OPM_SWEEP_COOPERATIVE) return OPM_ERR_ARG;
  if (o.small_phase_slices < -1) return OPM_ERR_ARG;
  if (o.cp_sweeps < 0 || o.cp_sweeps > kMaxCpSweeps || o.tri_sweeps < 0 || o.tri_sweeps > kMaxTriSweeps)
    return OPM_ERR_ARG;
  if (o.product_reuse != 0 && o.product_reuse != -1) return OPM_ERR_ARG;
  return OPM_OK;
}

// Fills the handle's per-call fields for a solve; stages host vectors.
opm_status prepare_solve(opm_solver *h, const double *b, double *x, double rtol, int32_t maxit, bool *x_dev) {
  const double *db = nullptr;
  opm_status s = staged_vec(h, b, &db);
  if (s != OPM_OK) return s;
  *x_dev = is_device_ptr(x);
  h->sys.b_in = db;
  h->sys.x_out = *x_dev ? x : h->vec_out;
  h->sys.rtol = rtol;
  h->sys.maxit = maxit;
  h->sys.vals_in = nullptr;
  return OPM_OK;
}

opm_status worst_status(opm_status a, opm_status b) {
  if (a < 0) return a;
  if (b < 0) return b;
  return a != OPM_OK ? a : b;
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
  opt->sweep_launch = OPM_SWEEP_AUTO;
}

const char *opm_status_str(opm_status s) {
  const int v = (int)s;
  if (v == 0) return kStatusText[0];
  if (v == 1) return kStatusText[1];
  if (v <= -1 && v >= -9) return kStatusText[1 - v];
  return "unknown status";
}

void opm_destroy(opm_handle h) {
  if (!h) return;
  if (h->run) runner_destroy(h->run);
  if (!h->allocs.empty() || !h->well_allocs.empty()) cudaStreamSynchronize(h->stream);
  dfree(h->allocs, h->stream);
  dfree(h->well_allocs, h->stream);
  if (h->gm_V) cudaFree(h->gm_V);
  if (h->gm_part) cudaFree(h->gm_part);
  if (h->gm_exec) cudaGraphExecDestroy(h->gm_exec);
  if (h->gm_state) cudaFree(h->gm_state);
  if (h->gm_hstate) cudaFreeHost(h->gm_hstate);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

// Adds a conditional node of the given type at the current point of the
// capture on cap (the capture then continues after it) and returns its body.
opm_status capture_conditional(cudaStream_t cap, cudaGraphConditionalHandle ch, cudaGraphConditionalNodeType type,
                               cudaGraph_t *body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = ch;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = cp.conditional.phGraph_out[0];
  return OPM_OK;
}

// The conditional handle of the graph being captured on cap.
opm_status capture_handle(cudaStream_t cap, cudaGraphConditionalHandle *ch) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  CK(cudaGraphConditionalHandleCreate(ch, g, 0, cudaGraphCondAssignDefault));
  return OPM_OK;
}

// Restarted GMRES(m), the steps of the oracle's orc_gmres in the same order,
// as one graph: the start (b gathered, r = b, x = 0, ||b||, v_0 = r / beta),
// a device-side while loop whose body is one Arnoldi step (v_j through the
// preconditioner and the operator, classical Gram-Schmidt twice, the norm,
// v_{j+1}, then the Hessenberg column, Givens rotations and g in one
// thread) with a conditional end-of-cycle branch (H y = g, x += inv(M) V y,
// r = b - A x, the restart test, v_0 = r / beta), and the end (relres from
// that branch's true residual, x back to the caller's order, zero on
// failure).  The host reads the outcome once.
opm_status gm_build(opm_solver *h) {
  Runner &R = *h->run;
  const Sys &S = h->sys;
  const int64_t n3 = 3ll * h->n;
  const int ntile = S.ntiles_s;
  const GmKernels gk = gm_rows_per_thread(h->n, R.sms);
  const int ntile_g = std::max(1, (int)((h->n + gk.rows - 1) / gk.rows));  // Gram-Schmidt tiles
  const int egrid = (int)std::min<int64_t>((n3 + 255) / 256, 152 * 8);
  double *V = h->gm_V;
  GmState *gs = h->gm_state;
  double *part = h->gm_part;
  cudaStream_t cap;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  opm_status s = OPM_OK;
  cudaGraph_t g = nullptr, body = nullptr, tail_body = nullptr;
  cudaGraphConditionalHandle ch_loop = 0, ch_end = 0;
  auto dots = [&](const double *Vb, int sel, const double *w, double *out) {
    gk.dots<<<ntile_g, 256, 0, cap>>>(n3, Vb, n3, gs, sel, w, part);
    k_gm_reduce_s<<<kGmMaxVec, 256, 0, cap>>>(part, ntile_g, gs, sel, out);
  };
  // out = A in - wells; applied: in = inv(M) w was just formed (the product
  // may take the application's sums)
  auto op = [&](int which, const double *in, double *out, bool applied) {
    if (R.has_wells) k_wells<<<1, 256, 0, cap>>>(R.B, which);
    if (applied && R.reuse) k_gm_operator<true><<<ntile, 256, 0, cap>>>(R.B, in, out);
    else k_gm_operator<false><<<ntile, 256, 0, cap>>>(R.B, in, out);
  };
  // ---- start, loop node, end
  if (cudaGraphCreate(&g, 0) != cudaSuccess ||
      cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    s = OPM_ERR_CUDA;
  if (s == OPM_OK) {
    k_gather<<<R.ntiles, 256, 0, cap>>>(R.B);
    k_gm_copy_s<<<egrid, 256, 0, cap>>>(n3, S.w, S.p);
    k_gm_copy_s<<<egrid, 256, 0, cap>>>(n3, S.w, S.r);
    if (cudaMemsetAsync(S.x, 0, sizeof(double) * (size_t)n3, cap) != cudaSuccess) s = OPM_ERR_CUDA;
    dots(S.r, 1, S.r, &gs->nrm2);
    s = capture_handle(cap, &ch_loop);
    if (s == OPM_OK) {
      k_gm_init<<<1, 1, 0, cap>>>(gs, ch_loop);
      k_gm_scale_s<<<egrid, 256, 0, cap>>>(n3, S.r, gs, 1, V, n3, S.w);
      s = capture_conditional(cap, ch_loop, cudaGraphCondTypeWhile, &body);
    }
    if (s == OPM_OK) {
      // the loop only ends after an end-of-cycle branch, whose last norm is
      // ||b - A x|| of the final x; without a cycle x = 0 and r = b
      k_gm_final<<<1, 1, 0, cap>>>(gs);
      k_gm_vec_s<<<egrid, 256, 0, cap>>>(n3, S.x, S.x, S.x, 2, gs);  // x = 0 on failure
      k_gm_copy_s<<<egrid, 256, 0, cap>>>(n3, S.x, S.t);
      k_scatter<<<R.ntiles, 256, 0, cap>>>(R.B);
    }
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess) s = OPM_ERR_CUDA;
  }
  // ---- loop body: one Arnoldi step, then the end-of-cycle branch
  if (s == OPM_OK) {
    if (cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
      s = OPM_ERR_CUDA;
    } else {
      launch_apply<kModePlain>(R, cap);                                    // t = inv(M) v_j (held in w)
      op(4, S.t, S.v, true);                                               // v = A t
      dots(V, 0, S.v, gs->h1);
      // first correction with the second pass's projections, second
      // correction with the norm: one pass over V and w fewer each
      gk.correct<<<ntile_g, 256, 0, cap>>>(n3, V, n3, gs, gs->h1, S.v, part);
      k_gm_reduce_s<<<kGmMaxVec, 256, 0, cap>>>(part, ntile_g, gs, 0, gs->h2);
      gk.correct_norm<<<ntile_g, 256, 0, cap>>>(n3, V, n3, gs, gs->h2, S.v, part);
      k_gm_reduce_s<<<kGmMaxVec, 256, 0, cap>>>(part, ntile_g, gs, 1, &gs->nrm2);
      k_gm_scale_s<<<egrid, 256, 0, cap>>>(n3, S.v, gs, 0, V, n3, S.w);  // v_{j+1}, also into w
      s = capture_handle(cap, &ch_end);
      if (s == OPM_OK) {
        k_gm_step<<<1, 1, 0, cap>>>(gs, ch_end);
        s = capture_conditional(cap, ch_end, cudaGraphCondTypeIf, &tail_body);
      }
      if (s == OPM_OK) k_gm_cond<<<1, 1, 0, cap>>>(gs, ch_loop);
      if (cudaStreamEndCapture(cap, &body) != cudaSuccess) s = OPM_ERR_CUDA;
    }
  }
  // ---- end of a cycle
  if (s == OPM_OK) {
    if (cudaStreamBeginCaptureToGraph(cap, tail_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
      s = OPM_ERR_CUDA;
    } else {
      k_gm_trisolve<<<1, 1, 0, cap>>>(gs);
      k_gm_combine_s<<<egrid, 256, 0, cap>>>(n3, V, n3, gs, gs->y, S.w, 1);  // w = V y
      launch_apply<kModePlain>(R, cap);                                       // t = inv(M) V y
      k_gm_vec_s<<<egrid, 256, 0, cap>>>(n3, S.t, S.t, S.x, 1, gs);           // x += t
      op(2, S.x, S.v, false);
      k_gm_vec_s<<<egrid, 256, 0, cap>>>(n3, S.p, S.v, S.r, 0, gs);           // r = b - A x
      dots(S.r, 1, S.r, &gs->nrm2);
      k_gm_restart<<<1, 1, 0, cap>>>(gs);
      k_gm_scale_s<<<egrid, 256, 0, cap>>>(n3, S.r, gs, 1, V, n3, S.w);        // v_0 = r / beta, also into w
      if (cudaStreamEndCapture(cap, &tail_body) != cudaSuccess) s = OPM_ERR_CUDA;
    }
  }
  if (s == OPM_OK && cudaGraphInstantiate(&h->gm_exec, g, 0) != cudaSuccess) s = OPM_ERR_CUDA;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (s != OPM_OK) {
    fprintf(stderr, "opm_bsr: GMRES graph construction failed: %s\n", cudaGetErrorString(cudaGetLastError()));
    cudaGetLastError();
    h->gm_exec = nullptr;
  }
  return s;
}

opm_status opm_gmres_solve(opm_handle h, const double *b, double *x, double rtol, int32_t maxit, int32_t restart,
                           int32_t *iters, double *relres) {
  if (!h || (h->n > 0 && (!b || !x)) || !(rtol >= 0.0) || maxit < 0 || restart < 0 || restart > kGmMaxVec - 1 ||
      h->async_pending)
    return OPM_ERR_ARG;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (h->n == 0) return OPM_OK;
  if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  const int m = restart > 0 ? restart : 30;
  bool x_dev = false;
  opm_status s = prepare_solve(h, b, x, rtol, maxit, &x_dev);
  if (s != OPM_OK) return s;
  Runner &R = *h->run;
  cudaStream_t st = h->stream;
  const int64_t n3 = 3ll * h->n;
  const size_t vbytes = sizeof(double) * (size_t)n3;
  const int ntile = h->sys.ntiles_s;
  // ---- buffers (kept for later calls; the basis grows with m)
  if (h->gm_m < m) {
    if (h->gm_exec) cudaGraphExecDestroy(h->gm_exec);
    h->gm_exec = nullptr;
    if (h->gm_V) cudaFree(h->gm_V);
    h->gm_V = nullptr;
    h->gm_m = 0;
    if (cudaMalloc(&h->gm_V, vbytes * (size_t)(m + 1)) != cudaSuccess) {
      cudaGetLastError();
      h->gm_V = nullptr;
      return OPM_ERR_OOM;
    }
    h->gm_m = m;
  }
  // each buffer on its own: one that failed before is retried, none is used unallocated
  if ((!h->gm_part && cudaMalloc(&h->gm_part, sizeof(double) * (size_t)ntile * kGmMaxVec) != cudaSuccess) ||
      (!h->gm_state && cudaMalloc(&h->gm_state, sizeof(GmState)) != cudaSuccess) ||
      (!h->gm_hstate && cudaMallocHost(&h->gm_hstate, sizeof(GmState)) != cudaSuccess)) {
    cudaGetLastError();
    return OPM_ERR_OOM;
  }
  if ((s = runner_push(R)) != OPM_OK) return s;
  if (h->gm_exec && (h->gm_exec_V != h->gm_V || h->gm_exec_wells != R.has_wells)) {
    cudaGraphExecDestroy(h->gm_exec);
    h->gm_exec = nullptr;
  }
  if (!h->gm_exec) {
    if ((s = gm_build(h)) != OPM_OK) return s;
    h->gm_exec_V = h->gm_V;
    h->gm_exec_wells = R.has_wells;
  }
  // ---- inputs, the solve, the outcome
  GmState *hs = h->gm_hstate;
  hs->tol = rtol;
  hs->m = m;
  hs->maxit = maxit;
  hs->status = OPM_OK;
  CK(cudaMemcpyAsync(h->gm_state, hs, offsetof(GmState, h1), cudaMemcpyHostToDevice, st));
  CK(cudaGraphLaunch(h->gm_exec, st));
  CK(cudaMemcpyAsync(hs, h->gm_state, offsetof(GmState, h1), cudaMemcpyDeviceToHost, st));
  if (!x_dev) CK(cudaMemcpyAsync(x, h->vec_out, vbytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (iters) *iters = hs->k;
  if (relres) *relres = hs->relres;
  return (opm_status)hs->status;
}

opm_status opm_set_wells(opm_handle h, int32_t nwells, const int32_t *wptr, const int32_t *cells, const double *B,
                         const double *C, const double *Dinv) {
  if (!h || nwells < 0 || h->async_pending) return OPM_ERR_ARG;
  if (nwells > 0 && (!wptr || !cells || !B || !C || !Dinv)) return OPM_ERR_ARG;
  // ---- host copies of the structure (host or device pointers) and checks
  std::vector<int32_t> hp, hc;
  if (nwells > 0) {
    hp.resize((size_t)nwells + 1);
    CK(cudaMemcpy(hp.data(), wptr, sizeof(int32_t) * hp.size(), cudaMemcpyDefault));
    if (hp[0] != 0) return OPM_ERR_ARG;
    for (int32_t w = 0; w < nwells; ++w)
      if (hp[w + 1] < hp[w]) return OPM_ERR_ARG;
    hc.resize((size_t)hp[nwells]);
    if (!hc.empty()) CK(cudaMemcpy(hc.data(), cells, sizeof(int32_t) * hc.size(), cudaMemcpyDefault));
    for (int32_t c : hc)
      if (c < 0 || c >= h->n) return OPM_ERR_ARG;
  }
  // ---- drop the previous wells (no kernel of this handle is in flight after the sync)
  CK(cudaStreamSynchronize(h->stream));
  dfree(h->well_allocs, h->stream);
  Sys &S = h->sys;
  S.nwells = 0;
  S.w_ptr = S.w_cell = S.w_of = S.w_rptr = S.w_rperf = nullptr;
  S.w_B = S.w_C = S.w_Dinv = nullptr;
  S.w_mask = nullptr;
  S.w_t2 = S.w_corr = nullptr;
  S.w_rows = nullptr;
  S.nwrows = 0;
  if (nwells == 0 || h->n == 0) return OPM_OK;
  // ---- schedule-order cells, well of each perforation, perforations by row
  const int32_t nperf = hp[nwells];
  const Analysis &an = h->an;
  std::vector<int32_t> pcell((size_t)nperf), wof((size_t)nperf), rptr((size_t)h->n + 1, 0), rperf((size_t)nperf);
  std::vector<uint32_t> mask((size_t)h->nslices, 0u);
  for (int32_t w = 0; w < nwells; ++w)
    for (int32_t p = hp[w]; p < hp[w + 1]; ++p) {
      pcell[p] = an.iperm[hc[p]];
      wof[p] = w;
      rptr[pcell[p] + 1]++;
      mask[pcell[p] / kWarp] |= 1u << (pcell[p] % kWarp);
    }
  for (int32_t i = 0; i < h->n; ++i) rptr[i + 1] += rptr[i];
  {
    std::vector<int32_t> fill(rptr.begin(), rptr.end() - 1);
    for (int32_t p = 0; p < nperf; ++p) rperf[fill[pcell[p]]++] = p;
  }
  int64_t bytes = 0;
  int32_t *d_ptr, *d_cell, *d_of, *d_rptr, *d_rperf;
  uint32_t *d_mask;
  double *d_B, *d_C, *d_D;
  opm_status s;
#define UPW(ptr, vec) \
  if ((s = upload(h->well_allocs, bytes, h->stream, &ptr, vec)) != OPM_OK) return s
  UPW(d_ptr, hp);
  UPW(d_cell, pcell);
  UPW(d_of, wof);
  UPW(d_rptr, rptr);
  UPW(d_rperf, rperf);
  UPW(d_mask, mask);
#undef UPW
  if ((s = dalloc(h->well_allocs, bytes, h->stream, &d_B, 12 * (size_t)std::max(nperf, 1))) != OPM_OK) return s;
  if ((s = dalloc(h->well_allocs, bytes, h->stream, &d_C, 12 * (size_t)std::max(nperf, 1))) != OPM_OK) return s;
  if ((s = dalloc(h->well_allocs, bytes, h->stream, &d_D, 16 * (size_t)nwells)) != OPM_OK) return s;
  double *d_t2, *d_corr;
  if ((s = dalloc(h->well_allocs, bytes, h->stream, &d_t2, 4 * (size_t)nwells)) != OPM_OK) return s;
  if ((s = dalloc(h->well_allocs, bytes, h->stream, &d_corr, 3 * (size_t)h->n)) != OPM_OK) return s;
  std::vector<int32_t> wrows;
  for (int32_t i = 0; i < h->n; ++i)
    if (rptr[i + 1] > rptr[i]) wrows.push_back(i);
  int32_t *d_wrows;
  if ((s = upload(h->well_allocs, bytes, h->stream, &d_wrows, wrows)) != OPM_OK) return s;
  if (nperf > 0) {
    CK(cudaMemcpyAsync(d_B, B, sizeof(double) * 12 * (size_t)nperf, cudaMemcpyDefault, h->stream));
    CK(cudaMemcpyAsync(d_C, C, sizeof(double) * 12 * (size_t)nperf, cudaMemcpyDefault, h->stream));
  }
  CK(cudaMemcpyAsync(d_D, Dinv, sizeof(double) * 16 * (size_t)nwells, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  S.w_ptr = d_ptr;
  S.w_cell = d_cell;
  S.w_of = d_of;
  S.w_rptr = d_rptr;
  S.w_rperf = d_rperf;
  S.w_mask = d_mask;
  S.w_B = d_B;
  S.w_C = d_C;
  S.w_Dinv = d_D;
  S.w_t2 = d_t2;
  S.w_corr = d_corr;
  S.w_rows = d_wrows;
  S.nwrows = (int32_t)wrows.size();
  S.nwells = nwells;
  return OPM_OK;
}

namespace {

// The device part of a new handle h whose analysis is done: h->an (kept =
// NULL) or a kept analysis, whose host part is copied into h->an.  Events,
// device memory, the uploaded analysis, the handle's batch of one and the
// first factorisation of vals.  Takes ownership of h.
opm_status finish_create(opm_solver *h, const Analysis *kept, const double *vals, const opm_options &o,
                         opm_handle *out) {
  auto fail = [&](opm_status s) {
    opm_destroy(h);
    return s;
  };
  if (kept) copy_host_part(h->an, *kept);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(OPM_ERR_CUDA);
  }
  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return fail(OPM_ERR_CUDA);
    }
  const int32_t nb = h->an.n;
  h->n = nb;
  h->nnzb = h->an.nnzb;
  h->nslices = (nb + kWarp - 1) / kWarp;
  h->ntiles = std::max(1, (nb + kTileRows - 1) / kTileRows);
  if (nb == 0) {
    h->factors_ok = true;
    *out = h;
    return OPM_OK;
  }
  opm_status s = alloc_system(h, kept ? *kept : h->an);
  if (!kept) drop_device_lists(h->an);
  if (s != OPM_OK) return fail(s);
  std::vector<opm_solver *> one{h};
  if ((s = runner_create(one, h->stream, o, &h->run)) != OPM_OK) return fail(s);
  s = factor_impl(h, vals);
  if (s == OPM_ERR_ZERO_PIVOT) {
    // the handle stays usable: the row can be read and new values factored
    *out = h;
    return s;
  }
  if (s != OPM_OK) return fail(s);
  *out = h;
  return OPM_OK;
}

// A host copy of a pattern given in host or device memory; rp, ci, pt point
// at the caller's arrays or at the copies.
opm_status host_pattern(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                        std::vector<int32_t> &hrp, std::vector<int32_t> &hci, std::vector<int32_t> &hpart,
                        const int32_t **rp, const int32_t **ci, const int32_t **pt) {
  *rp = rowptr;
  *ci = colidx;
  *pt = part;
  if (is_device_ptr(rowptr)) {
    hrp.resize((size_t)nb + 1);
    if (cudaMemcpy(hrp.data(), rowptr, sizeof(int32_t) * hrp.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OPM_ERR_CUDA;
    *rp = hrp.data();
  }
  const int64_t nnzb = (*rp)[nb];
  if (nnzb < 0) return OPM_ERR_PATTERN;
  if (nb > 0 && is_device_ptr(colidx)) {
    hci.resize((size_t)nnzb);
    if (cudaMemcpy(hci.data(), colidx, sizeof(int32_t) * hci.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OPM_ERR_CUDA;
    *ci = hci.data();
  }
  if (part && nb > 0 && is_device_ptr(part)) {
    hpart.resize((size_t)nb);
    if (cudaMemcpy(hpart.data(), part, sizeof(int32_t) * hpart.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OPM_ERR_CUDA;
    *pt = hpart.data();
  }
  return OPM_OK;
}

// Counts and permutation of an analysis for the caller.
void analysis_info(const Analysis &an, int32_t *perm, opm_analysis_info *info) {
  if (perm && an.n > 0) memcpy(perm, an.perm.data(), sizeof(int32_t) * (size_t)an.n);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->schedule = an.schedule;
    info->nsets = an.nsets;
    info->nphases = an.n > 0 ? (int32_t)an.phase_ptr.size() - 1 : 0;
    info->nnzb_kept = an.nnzb_kept;
    info->nnzb_lower = an.nnz_l;
    info->nnzb_upper = an.nnz_u;
    info->nupdates = an.nupd;
    info->rows_identity = an.rows_identity;
    info->nnzb_product = an.nnzb_product;
    info->rows_reuse = an.rows_reuse;
  }
}

opm_status new_handle(const opm_options *opt, opm_options *o, opm_solver **h) {
  opm_options_default(o);
  if (opt) *o = *opt;
  if (check_options(*o) != OPM_OK) return OPM_ERR_ARG;
  *h = new (std::nothrow) opm_solver();
  if (!*h) return OPM_ERR_OOM;
  (*h)->opt = *o;
  (*h)->stream = (cudaStream_t)o->stream;
  (*h)->fp32 = o->precision == OPM_PREC_FP32_FACTORS;
  return OPM_OK;
}

opm_status create_impl(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                       const int32_t *part, const opm_options *opt, opm_handle *out) {
  if (!out) return OPM_ERR_ARG;
  *out = nullptr;
  t_create_err_row = -1;
  if (nb < 0 || nb > OPM_MAX_ROWS || !rowptr || (nb > 0 && (!colidx || !vals))) return OPM_ERR_ARG;
  opm_options o;
  opm_solver *h = nullptr;
  opm_status s = new_handle(opt, &o, &h);
  if (s != OPM_OK) return s;
  std::vector<int32_t> hrp, hci, hpart;
  const int32_t *rp, *ci, *pt;
  if ((s = host_pattern(nb, rowptr, colidx, part, hrp, hci, hpart, &rp, &ci, &pt)) != OPM_OK) {
    opm_destroy(h);
    return s;
  }
  int32_t err_row = -1;
  s = analyse(nb, rp, ci, pt, o.schedule, h->an, &err_row);
  t_create_err_row = err_row;
  if (s != OPM_OK) {
    opm_destroy(h);
    return s;
  }
  return finish_create(h, nullptr, vals, o, out);
}

}  // namespace

opm_status opm_bsr_create(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                          const opm_options *opt, opm_handle *out) {
  return create_impl(nb, rowptr, colidx, vals, nullptr, opt, out);
}

opm_status opm_bsr_create_jacobi(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                                 const int32_t *part, const opm_options *opt, opm_handle *out) {
  if (out) *out = nullptr;
  if (nb > 0 && !part) return OPM_ERR_ARG;
  return create_impl(nb, rowptr, colidx, vals, part, opt, out);
}

opm_status opm_bsr_analyse(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                           int32_t schedule, int32_t *perm, opm_analysis_info *info) {
  t_create_err_row = -1;
  if (nb < 0 || nb > OPM_MAX_ROWS || !rowptr || (nb > 0 && !colidx) || schedule < OPM_SCHED_AUTO ||
      schedule > OPM_SCHED_COLOUR_KEMPE)
    return OPM_ERR_ARG;
  Analysis an;
  int32_t err_row = -1;
  const opm_status s = analyse(nb, rowptr, colidx, part, schedule, an, &err_row);
  t_create_err_row = err_row;
  if (s != OPM_OK) return s;
  analysis_info(an, perm, info);
  return OPM_OK;
}

opm_status opm_analysis_create(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                               int32_t schedule, opm_analysis *out) {
  if (!out) return OPM_ERR_ARG;
  *out = nullptr;
  t_create_err_row = -1;
  if (nb < 0 || nb > OPM_MAX_ROWS || !rowptr || (nb > 0 && !colidx) || schedule < OPM_SCHED_AUTO ||
      schedule > OPM_SCHED_COLOUR_KEMPE)
    return OPM_ERR_ARG;
  std::vector<int32_t> hrp, hci, hpart;
  const int32_t *rp, *ci, *pt;
  opm_status s = host_pattern(nb, rowptr, colidx, part, hrp, hci, hpart, &rp, &ci, &pt);
  if (s != OPM_OK) return s;
  opm_analysis a = new (std::nothrow) opm_analysis_s();
  if (!a) return OPM_ERR_OOM;
  int32_t err_row = -1;
  s = analyse(nb, rp, ci, pt, schedule, a->an, &err_row);
  t_create_err_row = err_row;
  if (s != OPM_OK) {
    delete a;
    return s;
  }
  *out = a;
  return OPM_OK;
}

opm_status opm_bsr_create_from_analysis(opm_analysis a, const double *vals, const opm_options *opt,
                                        opm_handle *out) {
  if (!out) return OPM_ERR_ARG;
  *out = nullptr;
  if (!a || (a->an.n > 0 && !vals)) return OPM_ERR_ARG;
  opm_options o;
  opm_solver *h = nullptr;
  opm_status s = new_handle(opt, &o, &h);
  if (s != OPM_OK) return s;
  return finish_create(h, &a->an, vals, o, out);
}

opm_status opm_analysis_get_info(opm_analysis a, int32_t *nb, int64_t *nnzb, int32_t *perm,
                                 opm_analysis_info *info) {
  if (!a) return OPM_ERR_ARG;
  if (nb) *nb = a->an.n;
  if (nnzb) *nnzb = a->an.nnzb;
  analysis_info(a->an, perm, info);
  return OPM_OK;
}

void opm_analysis_destroy(opm_analysis a) { delete a; }

opm_status opm_ilu0_factor(opm_handle h, const double *vals) {
  if (!h || h->async_pending) return OPM_ERR_ARG;
  return factor_impl(h, vals);
}

opm_status opm_bicgstab_solve(opm_handle h, const double *b, double *x, double rtol, int32_t maxit,
                              int32_t *iters, double *relres) {
  if (!h || (h->n > 0 && (!b || !x)) || !(rtol >= 0.0) || h->async_pending) return OPM_ERR_ARG;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (h->n == 0) return OPM_OK;
  if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  bool x_dev = false;
  opm_status s = prepare_solve(h, b, x, rtol, maxit, &x_dev);
  if (s != OPM_OK) return s;
  Runner &R = *h->run;
  const size_t vbytes = sizeof(double) * 3 * (size_t)h->n;
  CK(cudaEventRecord(h->ev[0], h->stream));
  if (R.profile) {
    if ((s = runner_solve_profiled(R, h->timing)) != OPM_OK) return s;
  } else {
    if ((s = runner_enqueue(R, false, true)) != OPM_OK) return s;
    if ((s = runner_wait(R)) != OPM_OK) return s;
    h->timing.launches += solve_graph_launches(R);
  }
  if (!x_dev) CK(cudaMemcpyAsync(x, h->vec_out, vbytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaEventRecord(h->ev[1], h->stream));
  CK(cudaEventSynchronize(h->ev[1]));
  cudaEventElapsedTime(&h->timing.iterate_ms, h->ev[0], h->ev[1]);
  h->timing.setup_ms = 0.f;
  h->timing.finish_ms = 0.f;
  const Result &r = R.h_res[0];
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  return (opm_status)r.status;
}

opm_status opm_solve_launch(opm_handle h, const double *vals, const double *b, double *x, double rtol,
                            int32_t maxit) {
  if (!h || h->n == 0 || !b || !x || !(rtol >= 0.0) || h->async_pending || h->run->profile) return OPM_ERR_ARG;
  if (!vals && !h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  const double *dv = nullptr;
  opm_status s = staged_vals(h, vals, &dv);
  if (s != OPM_OK) return s;
  bool x_dev = false;
  if ((s = prepare_solve(h, b, x, rtol, maxit, &x_dev)) != OPM_OK) return s;
  h->sys.vals_in = dv;
  Runner &R = *h->run;
  s = runner_enqueue(R, vals != nullptr, true);
  h->sys.vals_in = nullptr;
  if (s != OPM_OK) return s;
  if (!x_dev) {
    CK(cudaMemcpyAsync(x, h->vec_out, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(R.ev_done, h->stream));  // completion now includes the copy back
  }
  h->async_pending = true;
  h->timing.launches += vals ? h->run->factor_launches : 0;
  return OPM_OK;
}

int32_t opm_solve_ready(opm_handle h) {
  if (!h || !h->async_pending) return 1;
  const cudaError_t e = cudaEventQuery(h->run->ev_done);
  if (e == cudaErrorNotReady) return 0;
  cudaGetLastError();
  return 1;
}

opm_status opm_solve_wait(opm_handle h, int32_t *iters, double *relres) {
  if (!h || !h->async_pending) return OPM_ERR_ARG;
  Runner &R = *h->run;
  h->async_pending = false;
  opm_status s = runner_wait(R);
  if (s != OPM_OK) return s;
  const Result &r = R.h_res[0];
  h->timing.launches += solve_graph_launches(R);
  if (r.status == OPM_ERR_ZERO_PIVOT) {
    h->factors_ok = false;
    h->last_err_row = (r.err_row >= 0 && r.err_row < h->n) ? h->an.perm[r.err_row] : -1;
  } else {
    h->factors_ok = true;
  }
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  return (opm_status)r.status;
}

opm_status opm_spmv(opm_handle h, const double *x, double *y) {
  if (!h || (h->n > 0 && (!x || !y)) || h->async_pending) return OPM_ERR_ARG;
  if (h->n == 0) return OPM_OK;
  const double *dx = nullptr;
  opm_status s = staged_vec(h, x, &dx);
  if (s != OPM_OK) return s;
  const bool y_dev = is_device_ptr(y);
  h->sys.b_in = dx;
  h->sys.x_out = y_dev ? y : h->vec_out;
  Runner &R = *h->run;
  if ((s = runner_push(R)) != OPM_OK) return s;
  k_gather<<<R.ntiles, 256, 0, h->stream>>>(R.B);
  if (R.has_wells) k_wells<<<R.nsys, 256, 0, h->stream>>>(R.B, 3);
  k_spmv_plain<<<R.ntiles_s, 256, 0, h->stream>>>(R.B);
  CK(cudaGetLastError());
  h->timing.launches += 2;
  if (!y_dev)
    CK(cudaMemcpyAsync(y, h->vec_out, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OPM_OK;
}

opm_status opm_ilu_apply(opm_handle h, const double *r, double *z) {
  if (!h || (h->n > 0 && (!r || !z)) || h->async_pending) return OPM_ERR_ARG;
  if (h->n == 0) return OPM_OK;
  if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  const double *dr = nullptr;
  opm_status s = staged_vec(h, r, &dr);
  if (s != OPM_OK) return s;
  const bool z_dev = is_device_ptr(z);
  h->sys.b_in = dr;
  h->sys.x_out = z_dev ? z : h->vec_out;
  Runner &R = *h->run;
  if ((s = runner_push(R)) != OPM_OK) return s;
  k_gather<<<R.ntiles, 256, 0, h->stream>>>(R.B);
  const int nl = launch_apply<kModePlain>(R, h->stream);
  k_scatter<<<R.ntiles, 256, 0, h->stream>>>(R.B);
  k_results<<<results_blocks(R), 128, 0, h->stream>>>(R.B, R.d_res);
  CK(cudaGetLastError());
  h->timing.launches += 3 + nl;
  if (!z_dev)
    CK(cudaMemcpyAsync(z, h->vec_out, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  if ((s = runner_pull_results(R)) != OPM_OK) return s;
  CK(cudaStreamSynchronize(h->stream));
  // only an expired bounded wait can fail here
  if (R.h_res[0].status == OPM_ERR_TIMEOUT) return OPM_ERR_TIMEOUT;
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
  info->device_bytes = h->dev_bytes + (h->run ? h->run->dev_bytes : 0);
  info->nphases = h->n > 0 ? (int32_t)h->an.phase_ptr.size() - 1 : 0;
  info->rows_identity = h->an.rows_identity;
  info->nupdates = h->an.nupd;
  const bool reuse = product_reuse_applies(h->opt, h->fp32);
  info->nnzb_product = reuse ? h->an.nnzb_product : h->nnzb;
  info->rows_reuse = reuse ? h->an.rows_reuse : 0;
  info->reserved2 = 0;
  return OPM_OK;
}

opm_status opm_get_permutation(opm_handle h, int32_t *perm) {
  if (!h || (!perm && h->n > 0)) return OPM_ERR_ARG;
  if (h->n > 0) memcpy(perm, h->an.perm.data(), sizeof(int32_t) * (size_t)h->n);
  return OPM_OK;
}

opm_status opm_get_factors(opm_handle h, double *lu, double *dinv) {
  if (!h || h->async_pending) return OPM_ERR_ARG;
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
      if (slot < 0) {  // outside the preconditioner's pattern
        for (int e = 0; e < 9; ++e) lu[9 * c + e] = 0.0;
        continue;
      }
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

// ---------------------------------------------------------------- batches

void opm_batch_destroy(opm_batch b) {
  if (!b) return;
  if (b->run) runner_destroy(b->run);
  delete b;
}

opm_status opm_batch_create(int32_t nsys, const opm_handle *hs, const opm_options *opt, opm_batch *out) {
  if (!out) return OPM_ERR_ARG;
  *out = nullptr;
  if (nsys < 1 || !hs) return OPM_ERR_ARG;
  opm_options o;
  opm_options_default(&o);
  if (opt) o = *opt;
  if (check_options(o) != OPM_OK) return OPM_ERR_ARG;
  std::vector<opm_solver *> mem;
  for (int i = 0; i < nsys; ++i) {
    opm_solver *h = hs[i];
    if (!h || h->n == 0 || !h->run || h->fp32 != hs[0]->fp32 || h->device != hs[0]->device) return OPM_ERR_ARG;
    for (auto *m : mem)
      if (m == h) return OPM_ERR_ARG;
    mem.push_back(h);
  }
  opm_batch b = new (std::nothrow) opm_batch_s();
  if (!b) return OPM_ERR_OOM;
  b->members = mem;
  opm_options ob = o;
  ob.profile_kernels = 0;
  opm_status s = runner_create(mem, (cudaStream_t)o.stream, ob, &b->run);
  if (s != OPM_OK) {
    opm_batch_destroy(b);
    return s;
  }
  *out = b;
  return OPM_OK;
}

opm_status opm_batch_factor(opm_batch b, const double *const *vals, opm_status *st) {
  if (!b || b->async_pending) return OPM_ERR_ARG;
  Runner &R = *b->run;
  opm_status s;
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    if (h->async_pending) return OPM_ERR_ARG;
    const double *dv = nullptr;
    if ((s = staged_vals(h, vals ? vals[i] : nullptr, &dv)) != OPM_OK) return s;
    h->sys.vals_in = dv;
  }
  // host-to-device staging ran on the members' streams: complete it first
  for (auto *h : b->members) CK(cudaStreamSynchronize(h->stream));
  s = runner_enqueue(R, true, false);
  for (auto *h : b->members) h->sys.vals_in = nullptr;
  if (s != OPM_OK) return s;
  if ((s = runner_wait(R)) != OPM_OK) return s;
  opm_status worst = OPM_OK;
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    const Result &r = R.h_res[i];
    if (r.status < 0) {
      h->factors_ok = false;
      h->last_err_row = (r.err_row >= 0 && r.err_row < h->n) ? h->an.perm[r.err_row] : -1;
      if (st) st[i] = (opm_status)r.status;
      worst = worst_status(worst, (opm_status)r.status);
    } else {
      h->factors_ok = true;
      h->last_err_row = -1;
      if (st) st[i] = OPM_OK;
    }
  }
  return worst;
}

opm_status opm_batch_solve(opm_batch b, const double *const *bv, double *const *xv, const double *rtol,
                           int32_t maxit, int32_t *iters, double *relres, opm_status *st) {
  if (!b || !bv || !xv || b->async_pending) return OPM_ERR_ARG;
  Runner &R = *b->run;
  std::vector<char> x_dev(R.nsys);
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    if (!bv[i] || !xv[i] || h->async_pending) return OPM_ERR_ARG;
    const double rt = rtol ? rtol[i] : 1e-2;
    if (!(rt >= 0.0)) return OPM_ERR_ARG;
    if (!h->factors_ok) return OPM_ERR_ZERO_PIVOT;
    bool xd = false;
    opm_status s = prepare_solve(h, bv[i], xv[i], rt, maxit, &xd);
    if (s != OPM_OK) return s;
    x_dev[i] = xd;
  }
  for (auto *h : b->members) CK(cudaStreamSynchronize(h->stream));
  opm_status s = runner_enqueue(R, false, true);
  if (s != OPM_OK) return s;
  if ((s = runner_wait(R)) != OPM_OK) return s;
  opm_status worst = OPM_OK;
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    if (!x_dev[i]) CK(cudaMemcpy(xv[i], h->vec_out, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost));
    const Result &r = R.h_res[i];
    if (iters) iters[i] = r.iters;
    if (relres) relres[i] = r.relres;
    if (st) st[i] = (opm_status)r.status;
    worst = worst_status(worst, (opm_status)r.status);
  }
  return worst;
}

opm_status opm_batch_launch(opm_batch b, const double *const *vals, const double *const *bv, double *const *xv,
                            const double *rtol, int32_t maxit) {
  if (!b || !bv || !xv || b->async_pending) return OPM_ERR_ARG;
  Runner &R = *b->run;
  b->sat_out.assign(R.nsys, 0);
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    if (!bv[i] && !xv[i]) {  // sits this launch out
      b->sat_out[i] = 1;
      continue;
    }
    const double *v = vals ? vals[i] : nullptr;
    const double rt = rtol ? rtol[i] : 1e-2;
    if (!bv[i] || !xv[i] || !is_device_ptr(bv[i]) || !is_device_ptr(xv[i]) || (v && !is_device_ptr(v)) ||
        !(rt >= 0.0) || h->async_pending)
      return OPM_ERR_ARG;
    if (!vals && !h->factors_ok) return OPM_ERR_ZERO_PIVOT;
  }
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    const bool out = b->sat_out[i] != 0;
    h->sys.skip = out ? 1 : 0;
    h->sys.b_in = out ? nullptr : bv[i];
    h->sys.x_out = out ? nullptr : xv[i];
    h->sys.rtol = rtol ? rtol[i] : 1e-2;
    h->sys.maxit = maxit;
    h->sys.vals_in = (vals && !out) ? vals[i] : nullptr;
  }
  opm_status s = runner_enqueue(R, vals != nullptr, true);
  for (auto *h : b->members) {
    h->sys.vals_in = nullptr;
    h->sys.skip = 0;
  }
  if (s != OPM_OK) return s;
  b->async_pending = true;
  return OPM_OK;
}

int32_t opm_batch_ready(opm_batch b) {
  if (!b || !b->async_pending) return 1;
  const cudaError_t e = cudaEventQuery(b->run->ev_done);
  if (e == cudaErrorNotReady) return 0;
  cudaGetLastError();
  return 1;
}

opm_status opm_batch_wait(opm_batch b, int32_t *iters, double *relres, opm_status *st) {
  if (!b || !b->async_pending) return OPM_ERR_ARG;
  Runner &R = *b->run;
  b->async_pending = false;
  opm_status s = runner_wait(R);
  if (s != OPM_OK) return s;
  opm_status worst = OPM_OK;
  for (int i = 0; i < R.nsys; ++i) {
    opm_solver *h = b->members[i];
    if (!b->sat_out.empty() && b->sat_out[i]) {
      if (iters) iters[i] = 0;
      if (relres) relres[i] = 0.0;
      if (st) st[i] = OPM_OK;
      continue;
    }
    const Result &r = R.h_res[i];
    h->factors_ok = r.status != OPM_ERR_ZERO_PIVOT;
    if (iters) iters[i] = r.iters;
    if (relres) relres[i] = r.relres;
    if (st) st[i] = (opm_status)r.status;
    worst = worst_status(worst, (opm_status)r.status);
  }
  return worst;
}

}  // extern "C"
