// Autotuner of the launch configuration (schedule, sweep launch, iterations
// per loop body, small-phase threshold): times refactorisation + solve of
// each candidate through the public entry points and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opm_bsr.h"

namespace {

struct Cand {
  int32_t schedule, sweep, chunk, small;
};

// A run of one candidate: create() builds its handles (untimed), run() does
// one refactorisation + solve and reports status and iterations, destroy()
// frees everything.
struct Problem {
  virtual ~Problem() = default;
  virtual opm_status create(const opm_options &o, int32_t *max_phases) = 0;
  virtual opm_status run(opm_status *st, int32_t *iters) = 0;
  virtual void destroy() = 0;
};

int status_class(int32_t s) { return s == OPM_OK ? 0 : s == OPM_NOT_CONVERGED ? 1 : 2; }

double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  const size_t m = v.size() / 2;
  return v.size() % 2 ? v[m] : 0.5 * (v[m - 1] + v[m]);
}

// Times one candidate; returns false when it could not be built or run.
bool time_candidate(Problem &P, const opm_options &o, int repeats, opm_tune_entry &e, int32_t *max_phases,
                    opm_status *first_err) {
  e.schedule = o.schedule;
  e.sweep_launch = o.sweep_launch;
  e.chunk = o.chunk;
  e.small_phase_slices = o.small_phase_slices;
  e.ms = -1.0;
  e.iters = 0;
  opm_status s = P.create(o, max_phases);
  if (s != OPM_OK) {
    *max_phases = INT_MAX;
    e.status = (int32_t)s;
    if (*first_err == OPM_OK) *first_err = s;
    P.destroy();
    return false;
  }
  opm_status st = OPM_OK;
  int32_t it = 0;
  s = P.run(&st, &it);  // warm-up
  std::vector<double> ms;
  for (int r = 0; r < repeats && status_class(s) < 2; ++r) {
    const auto t0 = std::chrono::steady_clock::now();
    s = P.run(&st, &it);
    const auto t1 = std::chrono::steady_clock::now();
    ms.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
  }
  P.destroy();
  e.status = status_class(s) < 2 ? (int32_t)st : (int32_t)s;
  e.iters = it;
  if (status_class(e.status) == 2) {
    if (*first_err == OPM_OK) *first_err = (opm_status)e.status;
    return false;
  }
  e.ms = median(ms);
  return true;
}

bool better(const opm_tune_entry &a, const opm_tune_entry &b) {
  const int ca = status_class(a.status), cb = status_class(b.status);
  if (ca != cb) return ca < cb;
  return a.ms < b.ms;
}

opm_status tune(Problem &P, bool allow_natural, int32_t repeats, const opm_options *base, opm_options *best,
                opm_tune_report *report) {
  opm_options o0;
  opm_options_default(&o0);
  if (base) o0 = *base;
  o0.profile_kernels = 0;
  o0.debug_skip_item = -1;
  if (repeats < 1) repeats = 3;
  opm_tune_report rep;
  memset(&rep, 0, sizeof(rep));
  rep.best = -1;
  opm_status first_err = OPM_OK;
  // runs one candidate; returns the largest phase count of its systems
  auto tryc = [&](const Cand &c) -> int32_t {
    if (rep.ncand >= OPM_TUNE_MAX) return INT_MAX;
    opm_options o = o0;
    o.schedule = c.schedule;
    o.sweep_launch = c.sweep;
    o.chunk = c.chunk;
    o.small_phase_slices = c.small;
    int32_t phases = INT_MAX;
    opm_tune_entry &e = rep.cand[rep.ncand++];
    if (time_candidate(P, o, repeats, e, &phases, &first_err) &&
        (rep.best < 0 || better(e, rep.cand[rep.best])))
      rep.best = rep.ncand - 1;
    return phases;
  };
  // 1. schedule x sweep launch (one launch per phase only for few phases)
  std::vector<int32_t> scheds = {OPM_SCHED_LEVEL, OPM_SCHED_COLOUR, OPM_SCHED_COLOUR_SL, OPM_SCHED_COLOUR_KEMPE};
  if (allow_natural) scheds.push_back(OPM_SCHED_NATURAL);
  for (int32_t sc : scheds) {
    const int32_t phases = tryc({sc, OPM_SWEEP_COOPERATIVE, 2, 0});
    if (phases <= 1024) tryc({sc, OPM_SWEEP_PER_PHASE, 2, 0});
  }
  // 2. iterations per loop body
  if (rep.best >= 0) {
    const opm_tune_entry b = rep.cand[rep.best];
    for (int32_t ch : {1, 4}) tryc({b.schedule, b.sweep_launch, ch, b.small_phase_slices});
  }
  // 3. small-phase threshold of the per-phase launches
  if (rep.best >= 0 && rep.cand[rep.best].sweep_launch == OPM_SWEEP_PER_PHASE) {
    const opm_tune_entry b = rep.cand[rep.best];
    for (int32_t sm : {-1, 1 << 30}) tryc({b.schedule, b.sweep_launch, b.chunk, sm});
  }
  if (best) {
    *best = o0;
    if (rep.best >= 0) {
      const opm_tune_entry &b = rep.cand[rep.best];
      best->schedule = b.schedule;
      best->sweep_launch = b.sweep_launch;
      best->chunk = b.chunk;
      best->small_phase_slices = b.small_phase_slices;
    }
  }
  if (report) *report = rep;
  if (rep.best < 0) return first_err != OPM_OK ? first_err : OPM_ERR_ARG;
  return status_class(rep.cand[rep.best].status) == 0 ? OPM_OK : OPM_NOT_CONVERGED;
}

struct Single : Problem {
  int32_t nb;
  const int32_t *rowptr, *colidx;
  const double *vals, *b;
  double rtol;
  int32_t maxit;
  double *x = nullptr;
  opm_handle h = nullptr;
  opm_status create(const opm_options &o, int32_t *max_phases) override {
    if (!x && cudaMalloc(&x, sizeof(double) * 3 * (size_t)std::max(nb, 1)) != cudaSuccess) {
      cudaGetLastError();
      x = nullptr;
      return OPM_ERR_OOM;
    }
    opm_status s = opm_bsr_create(nb, rowptr, colidx, vals, &o, &h);
    if (s != OPM_OK) return s;
    opm_info info;
    if ((s = opm_get_info(h, &info)) != OPM_OK) return s;
    *max_phases = info.nphases;
    return OPM_OK;
  }
  opm_status run(opm_status *st, int32_t *iters) override {
    opm_status s = opm_ilu0_factor(h, vals);
    if (s != OPM_OK) return s;
    double rr = 0.0;
    *st = opm_bicgstab_solve(h, b, x, rtol, maxit, iters, &rr);
    return *st < 0 ? *st : OPM_OK;
  }
  void destroy() override {
    if (h) opm_destroy(h);
    h = nullptr;
  }
  ~Single() override {
    destroy();
    if (x) cudaFree(x);
  }
};

struct Multi : Problem {
  int32_t nsys;
  const int32_t *nb;
  const int32_t *const *rowptr, *const *colidx;
  const double *const *vals, *const *b;
  std::vector<double> rtol;
  int32_t maxit;
  double *xbuf = nullptr;
  std::vector<double *> x;
  std::vector<opm_handle> hs;
  opm_batch bt = nullptr;
  opm_status create(const opm_options &o, int32_t *max_phases) override {
    if (!xbuf) {
      size_t tot = 0;
      for (int32_t i = 0; i < nsys; ++i) tot += 3 * (size_t)nb[i];
      if (cudaMalloc(&xbuf, sizeof(double) * std::max<size_t>(tot, 1)) != cudaSuccess) {
        cudaGetLastError();
        xbuf = nullptr;
        return OPM_ERR_OOM;
      }
      x.resize(nsys);
      size_t off = 0;
      for (int32_t i = 0; i < nsys; ++i) {
        x[i] = xbuf + off;
        off += 3 * (size_t)nb[i];
      }
    }
    *max_phases = 0;
    for (int32_t i = 0; i < nsys; ++i) {
      opm_handle h = nullptr;
      opm_status s = opm_bsr_create(nb[i], rowptr[i], colidx[i], vals[i], &o, &h);
      if (h) hs.push_back(h);
      if (s != OPM_OK) return s;
      opm_info info;
      if ((s = opm_get_info(h, &info)) != OPM_OK) return s;
      *max_phases = std::max(*max_phases, info.nphases);
    }
    return opm_batch_create(nsys, hs.data(), &o, &bt);
  }
  opm_status run(opm_status *st, int32_t *iters) override {
    std::vector<opm_status> sts(nsys);
    std::vector<int32_t> its(nsys);
    opm_status s = opm_batch_factor(bt, vals, sts.data());
    if (s < 0) return s;
    s = opm_batch_solve(bt, b, x.data(), rtol.data(), maxit, its.data(), nullptr, sts.data());
    *st = s;
    *iters = *std::max_element(its.begin(), its.end());
    return s < 0 ? s : OPM_OK;
  }
  void destroy() override {
    if (bt) opm_batch_destroy(bt);
    bt = nullptr;
    for (opm_handle h : hs) opm_destroy(h);
    hs.clear();
  }
  ~Multi() override {
    destroy();
    if (xbuf) cudaFree(xbuf);
  }
};

// Report and options for a call rejected before any candidate ran.
opm_status rejected(const opm_options *base, opm_options *best, opm_tune_report *report) {
  if (report) {
    memset(report, 0, sizeof(*report));
    report->best = -1;
  }
  if (best) {
    if (base) *best = *base;
    else opm_options_default(best);
  }
  return OPM_ERR_ARG;
}

}  // namespace

extern "C" opm_status opm_autotune(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                                   const double *b, double rtol, int32_t maxit, int32_t repeats,
                                   const opm_options *base, opm_options *best, opm_tune_report *report) {
  if (nb < 0 || (nb > 0 && (!rowptr || !colidx || !vals || !b)) || !(rtol >= 0.0) || maxit < 0)
    return rejected(base, best, report);
  Single P;
  P.nb = nb;
  P.rowptr = rowptr;
  P.colidx = colidx;
  P.vals = vals;
  P.b = b;
  P.rtol = rtol;
  P.maxit = maxit;
  return tune(P, nb <= 4096, repeats, base, best, report);
}

extern "C" opm_status opm_autotune_batch(int32_t nsys, const int32_t *nb, const int32_t *const *rowptr,
                                         const int32_t *const *colidx, const double *const *vals,
                                         const double *const *b, const double *rtol, int32_t maxit,
                                         int32_t repeats, const opm_options *base, opm_options *best,
                                         opm_tune_report *report) {
  if (nsys < 1 || !nb || !rowptr || !colidx || !vals || !b || maxit < 0) return rejected(base, best, report);
  Multi P;
  P.nsys = nsys;
  P.nb = nb;
  P.rowptr = rowptr;
  P.colidx = colidx;
  P.vals = vals;
  P.b = b;
  P.maxit = maxit;
  P.rtol.assign(nsys, 1e-2);
  bool small = true;
  for (int32_t i = 0; i < nsys; ++i) {
    if (nb[i] < 0) return rejected(base, best, report);
    if (rtol) P.rtol[i] = rtol[i];
    small = small && nb[i] <= 4096;
  }
  return tune(P, small, repeats, base, best, report);
}
