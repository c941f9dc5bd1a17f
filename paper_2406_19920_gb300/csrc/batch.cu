// batch.cu -- the autotuner and batched solves of many independent grids.
//
// Autotuner.  For a grid shape and precision it times every available
// variant of the solve -- pencil kernel (two-ended sweep on a shared tile,
// the streaming two-ended sweep, or the warp-parallel substructured solve) x
// plane mode (split x and z passes, one CTA per y-plane, a cluster of C
// CTAs per plane, or tensor-core DFT products) -- on scratch buffers, keeps
// the fastest, and remembers it for the process (optionally in the text
// file named by IBM_TUNE_CACHE, one line per shape).  IBM_TUNE_DFT=0 leaves
// the tensor-core DFT mode out of the candidates (CUDA-core FFTs only).
//
// Batch.  ibm_batch_create makes one plan per instance (each with its own
// workspace, so instances never share scratch) and tunes every distinct
// shape.  ibm_batch_poisson captures all instances' solves into one CUDA
// graph -- a fork over K concurrent branches of the caller's stream, each
// branch running a share of the instances, largest first -- and replays it
// as a single graph launch.  K is tuned on the first call by timing the
// candidate graphs; graphs are cached per set of field pointers.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "plan.h"

namespace ibm {

struct TuneKey {
  int nx, ny, nz, precision, refine, dft;  // dft: the tensor-core DFT mode was a candidate
  bool operator<(const TuneKey &o) const {
    return std::tie(nx, ny, nz, precision, refine, dft) < std::tie(o.nx, o.ny, o.nz, o.precision, o.refine, o.dft);
  }
};

static bool tune_dft_allowed() {
  const char *e = getenv("IBM_TUNE_DFT");
  return !(e && atoi(e) == 0);
}
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune;
static bool g_tune_loaded = false;

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("IBM_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  TuneKey k;
  TuneChoice c;
  while (fscanf(f, "%d %d %d %d %d %d %d %d %lf", &k.nx, &k.ny, &k.nz, &k.precision, &k.refine, &k.dft,
                &c.pencil_mode, &c.use_plane, &c.ms) == 9)
    g_tune[k] = c;
  fclose(f);
}

static void tune_save_locked() {
  const char *path = getenv("IBM_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "w");
  if (!f) return;
  for (auto &kv : g_tune)
    fprintf(f, "%d %d %d %d %d %d %d %d %.6f\n", kv.first.nx, kv.first.ny, kv.first.nz, kv.first.precision,
            kv.first.refine, kv.first.dft, kv.second.pencil_mode, kv.second.use_plane, kv.second.ms);
  fclose(f);
}

static bool substructured_available(const ibm_plan_s *p) {
  const int n = p->ny;  // Poisson pencils (cell-centred)
  return p->precision == IBM_FP32_REFINED ? n <= 256 : n <= 128;
}

static bool segmented_available(const ibm_plan_s *p) {
  return p->precision == IBM_FP32_REFINED ? p->ny <= 512 : p->ny <= 256;
}

static int plane_candidates(const ibm_plan_s *p, int *modes) {
  int n = p->precision == IBM_FP64 ? plane_modes<double>(p->nx, p->nz, modes) : plane_modes<float>(p->nx, p->nz, modes);
  if (!tune_dft_allowed()) n = (int)(std::remove(modes, modes + n, kPlaneDft) - modes);
  return n;
}

// Times the Poisson solve of plan p for every variant and applies the
// fastest to p.  Synchronises the device; allocates two scratch fields.
int tune_plan(ibm_plan_s *p, TuneChoice *out) {
  const TuneKey key{p->nx, p->ny, p->nz, p->precision, p->refine, tune_dft_allowed() ? 1 : 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      p->pencil_mode = it->second.pencil_mode;
      p->use_plane = it->second.use_plane;
      // make sure every kernel of the chosen variant has its attributes set
      // before any stream capture: run it once
      void *a = nullptr, *b = nullptr;
      IBM_CUDA_TRY(cudaMalloc(&a, p->npts * p->esz));
      cudaError_t e = cudaMalloc(&b, p->npts * p->esz);
      if (e != cudaSuccess) { cudaFree(a); return cuda_error(e, "tuner scratch"); }
      cudaMemset(a, 0, p->npts * p->esz);
      int rc = plan_solve(p, 0, 0.0, 0, a, b, nullptr, 0, nullptr);
      cudaDeviceSynchronize();
      cudaFree(a);
      cudaFree(b);
      if (out) *out = it->second;
      return rc;
    }
  }
  void *a = nullptr, *b = nullptr;
  IBM_CUDA_TRY(cudaMalloc(&a, p->npts * p->esz));
  cudaError_t e = cudaMalloc(&b, p->npts * p->esz);
  if (e != cudaSuccess) { cudaFree(a); return cuda_error(e, "tuner scratch"); }
  cudaMemset(a, 0, p->npts * p->esz);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  TuneChoice best{0, p->use_plane, 1e30};
  int modes[8];
  const int nmodes = plane_candidates(p, modes);
  int rc = IBM_OK;
  int pms[4], npm = 0;
  if (segmented_available(p)) pms[npm++] = 4;
  pms[npm++] = 2;
  pms[npm++] = 3;
  if (substructured_available(p)) pms[npm++] = 1;
  for (int ip = 0; ip < npm && rc == IBM_OK; ++ip) {
    const int pm = pms[ip];
    for (int m = 0; m < nmodes && rc == IBM_OK; ++m) {
      const int up = modes[m];
      p->pencil_mode = pm;
      p->use_plane = up;
      for (int w = 0; w < 2 && rc == IBM_OK; ++w) rc = plan_solve(p, 0, 0.0, 0, a, b, nullptr, 0, nullptr);
      const int reps = 5;
      cudaEventRecord(e0, 0);
      for (int r = 0; r < reps && rc == IBM_OK; ++r) rc = plan_solve(p, 0, 0.0, 0, a, b, nullptr, 0, nullptr);
      cudaEventRecord(e1, 0);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (rc == IBM_OK && ms < best.ms) best = {pm, up, ms};
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  if (rc) return rc;
  p->pencil_mode = best.pencil_mode;
  p->use_plane = best.use_plane;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best;
    tune_save_locked();
  }
  if (out) *out = best;
  return IBM_OK;
}

}  // namespace ibm

using namespace ibm;

struct ibm_batch_s {
  int count = 0;
  std::vector<ibm_plan_s *> plans;
  std::vector<int> order;  // instances, largest grid first
  int branches = 0;        // graph fork width, tuned on the first call
  static constexpr int kMaxBranches = 16;
  cudaStream_t cap = nullptr;                 // graphs are captured and launched here
  cudaStream_t side[kMaxBranches] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxBranches] = {};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // order cap after / before the caller's stream
  struct Graph {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;  // most recently used last
  std::vector<Graph> stage_graphs;  // RK-stage graphs (instances with still markers), most recently used last
};

static void batch_free(ibm_batch_s *b) {
  if (!b) return;
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  for (auto &g : b->stage_graphs) cudaGraphExecDestroy(g.exec);
  for (auto *p : b->plans)
    if (p) ibm_plan_destroy(p);
  for (int k = 0; k < ibm_batch_s::kMaxBranches; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Captures the whole batch as one graph with K branches forked from `st`.
static int capture_batch(ibm_batch_s *b, int K, const void *const *rhs, void *const *phi, cudaStream_t st,
                         cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  IBM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = IBM_OK;
  cudaError_t e = cudaEventRecord(b->ev_fork, st);
  for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
  if (e != cudaSuccess) rc = cuda_error(e, "batch fork");
  for (size_t n = 0; n < b->order.size() && rc == IBM_OK; ++n) {
    const int i = b->order[n];
    rc = plan_solve(b->plans[i], 0, 0.0, 0, rhs[i], phi[i], nullptr, b->side[n % K], nullptr);
  }
  for (int k = 0; k < K && rc == IBM_OK; ++k) {
    e = cudaEventRecord(b->ev_join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join[k], 0);
    if (e != cudaSuccess) rc = cuda_error(e, "batch join");
  }
  e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
  return IBM_OK;
}

// Captures one RK stage of every instance as one graph with K branches.
static int capture_stage(ibm_batch_s *b, int K, ibm_state *states, ibm_markers *markers, int rk_stage, double dt,
                         double nu, cudaStream_t st, cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  IBM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = IBM_OK;
  cudaError_t e = cudaEventRecord(b->ev_fork, st);
  for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
  if (e != cudaSuccess) rc = cuda_error(e, "batch fork");
  for (size_t n = 0; n < b->order.size() && rc == IBM_OK; ++n) {
    const int i = b->order[n];
    ibm_markers *mk = markers && markers[i].n > 0 ? &markers[i] : nullptr;
    rc = substep_checked(b->plans[i], &states[i], rk_stage, dt, nu, mk, b->side[n % K]);
  }
  for (int k = 0; k < K && rc == IBM_OK; ++k) {
    e = cudaEventRecord(b->ev_join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join[k], 0);
    if (e != cudaSuccess) rc = cuda_error(e, "batch join");
  }
  e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
  return IBM_OK;
}

extern "C" {

int ibm_batch_create(int count, const int *dims, const double *h, int precision, int refine_iters,
                     ibm_batch *out) {
  if (!out || !dims || !h || count <= 0 || count > 4096)
    return set_error(IBM_ERR_ARG, "ibm_batch_create: bad arguments (count %d)", count);
  *out = nullptr;
  ibm_batch_s *b = new (std::nothrow) ibm_batch_s();
  if (!b) return set_error(IBM_ERR_OOM, "ibm_batch_create: host allocation");
  b->count = count;
  b->plans.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    int rc = ibm_plan_create(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], IBM_BC_PXZ_WALL_Y, h + 3 * i, precision,
                             refine_iters, &b->plans[i]);
    if (rc) {
      batch_free(b);
      return rc;
    }
  }
  // tune every distinct shape once; plans of the same shape share the choice
  std::map<TuneKey, TuneChoice> chosen;
  for (int i = 0; i < count; ++i) {
    ibm_plan_s *p = b->plans[i];
    const TuneKey k{p->nx, p->ny, p->nz, p->precision, p->refine, tune_dft_allowed() ? 1 : 0};
    auto it = chosen.find(k);
    if (it == chosen.end()) {
      TuneChoice c;
      int rc = tune_plan(p, &c);
      if (rc) {
        batch_free(b);
        return rc;
      }
      it = chosen.emplace(k, c).first;
    }
    p->pencil_mode = it->second.pencil_mode;
    p->use_plane = it->second.use_plane;
  }
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return b->plans[x]->npts > b->plans[y]->npts; });
  for (int k = 0; k < ibm_batch_s::kMaxBranches; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      batch_free(b);
      return cuda_error(e, "ibm_batch_create: streams");
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_error(e, "ibm_batch_create: event");
  }
  *out = b;
  return IBM_OK;
}

int ibm_batch_destroy(ibm_batch batch) {
  if (!batch) return set_error(IBM_ERR_ARG, "ibm_batch_destroy: NULL batch");
  cudaDeviceSynchronize();
  batch_free(batch);
  return IBM_OK;
}

int ibm_batch_poisson(ibm_batch b, const void *const *rhs, void *const *phi, void *stream) {
  if (!b || !rhs || !phi) return set_error(IBM_ERR_ARG, "ibm_batch_poisson: NULL argument");
  std::vector<uintptr_t> key(2 * (size_t)b->count);
  for (int i = 0; i < b->count; ++i) {
    if (!rhs[i] || !phi[i] || !aligned_to(rhs[i], 16) || !aligned_to(phi[i], 16))
      return set_error(IBM_ERR_ARG, "ibm_batch_poisson: field %d NULL or not 16-byte aligned", i);
    key[2 * i] = (uintptr_t)rhs[i];
    key[2 * i + 1] = (uintptr_t)phi[i];
  }
  // the graph runs on the batch's own stream, ordered after the caller's
  // stream and before its later work (capture cannot start on the legacy
  // default stream, which callers often use)
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t st = b->cap;
  IBM_CUDA_TRY(cudaEventRecord(b->ev_in, user));
  IBM_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_in, 0));
  for (size_t g = 0; g < b->graphs.size(); ++g) {
    if (b->graphs[g].key == key) {
      auto hit = b->graphs[g];
      b->graphs.erase(b->graphs.begin() + g);
      b->graphs.push_back(hit);
      IBM_CUDA_TRY(cudaGraphLaunch(hit.exec, st));
      IBM_CUDA_TRY(cudaEventRecord(b->ev_out, st));
      IBM_CUDA_TRY(cudaStreamWaitEvent(user, b->ev_out, 0));
      return IBM_OK;
    }
  }
  if (b->branches == 0) {
    // first call: time the candidate fork widths on scratch fields (repeated
    // launches must not touch the caller's data, which may be in place)
    std::vector<void *> tmp(2 * (size_t)b->count, nullptr);
    int rc = IBM_OK;
    for (int i = 0; i < b->count && rc == IBM_OK; ++i) {
      const size_t bytes = b->plans[i]->npts * b->plans[i]->esz;
      cudaError_t e1 = cudaMalloc(&tmp[2 * i], bytes);
      if (e1 == cudaSuccess) e1 = cudaMalloc(&tmp[2 * i + 1], bytes);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(tmp[2 * i], 0, bytes, st);
      if (e1 != cudaSuccess) rc = cuda_error(e1, "ibm_batch_poisson: tuning scratch");
    }
    std::vector<const void *> trhs(b->count);
    std::vector<void *> tphi(b->count);
    for (int i = 0; i < b->count; ++i) {
      trhs[i] = tmp[2 * i];
      tphi[i] = tmp[2 * i + 1];
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == IBM_OK) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
    float best = 1e30f;
    for (int K : {1, 2, 4, 8, 16}) {
      if (rc || (K > b->count && K > 1)) break;
      cudaGraphExec_t ex = nullptr;
      rc = capture_batch(b, K, trhs.data(), tphi.data(), st, &ex);
      if (rc) break;
      cudaGraphLaunch(ex, st);  // warm
      cudaEventRecord(e0, st);
      cudaGraphLaunch(ex, st);
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      cudaGraphExecDestroy(ex);
      if (e != cudaSuccess) {
        rc = cuda_error(e, "ibm_batch_poisson: tuning launch");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        b->branches = K;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    for (void *t : tmp)
      if (t) cudaFree(t);
    if (rc) {
      b->branches = 0;
      return rc;
    }
  }
  cudaGraphExec_t exec = nullptr;
  {
    int rc = capture_batch(b, b->branches, rhs, phi, st, &exec);
    if (rc) return rc;
  }
  if (b->graphs.size() >= 16) {
    cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back({key, exec});
  IBM_CUDA_TRY(cudaGraphLaunch(exec, st));
  IBM_CUDA_TRY(cudaEventRecord(b->ev_out, st));
  IBM_CUDA_TRY(cudaStreamWaitEvent(user, b->ev_out, 0));
  return IBM_OK;
}

int ibm_batch_substep(ibm_batch b, ibm_state *states, ibm_markers *markers, int rk_stage, double dt, double nu,
                      void *stream) {
  if (!b || !states) return set_error(IBM_ERR_ARG, "ibm_batch_substep: NULL argument");
  if (rk_stage < 1 || rk_stage > 3) return set_error(IBM_ERR_ARG, "ibm_batch_substep: rk_stage %d", rk_stage);
  if (!(dt > 0) || !(nu > 0)) return set_error(IBM_ERR_ARG, "ibm_batch_substep: dt and nu must be > 0");
  // every buffer a stage uses exists before any capture; the graph can be
  // replayed only when no instance's markers move (their positions are
  // evaluated on the host at capture)
  bool still = true;
  std::vector<uintptr_t> key;
  key.reserve(12 * (size_t)b->count + 3);
  key.push_back((uintptr_t)rk_stage);
  uint64_t bits[2];
  std::memcpy(&bits[0], &dt, 8);
  std::memcpy(&bits[1], &nu, 8);
  key.push_back((uintptr_t)bits[0]);
  key.push_back((uintptr_t)bits[1]);
  for (int i = 0; i < b->count; ++i) {
    const ibm_markers *mk = markers ? &markers[i] : nullptr;
    const int nmk = mk ? mk->n : 0;
    if (nmk < 0) return set_error(IBM_ERR_ARG, "ibm_batch_substep: instance %d: negative marker count", i);
    if (nmk > 0 && mk->motion != IBM_MOTION_STATIC) still = false;
    int rc = prepare_substep(b->plans[i], nmk);
    if (rc) return rc;
    const ibm_state &s = states[i];
    for (const void *f : {s.u, s.v, s.w, s.p, s.Nu, s.Nv, s.Nw}) key.push_back((uintptr_t)f);
    key.push_back((uintptr_t)nmk);
    if (nmk > 0)
      for (const void *f : {mk->X0, mk->dV, (const void *)mk->X, (const void *)mk->Ud, (const void *)mk->F})
        key.push_back((uintptr_t)f);
  }
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t st = b->cap;
  IBM_CUDA_TRY(cudaEventRecord(b->ev_in, user));
  IBM_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_in, 0));
  auto launch = [&](cudaGraphExec_t ex) -> int {
    IBM_CUDA_TRY(cudaGraphLaunch(ex, st));
    IBM_CUDA_TRY(cudaEventRecord(b->ev_out, st));
    IBM_CUDA_TRY(cudaStreamWaitEvent(user, b->ev_out, 0));
    return IBM_OK;
  };
  if (still) {
    for (size_t g = 0; g < b->stage_graphs.size(); ++g) {
      if (b->stage_graphs[g].key == key) {
        auto hit = b->stage_graphs[g];
        b->stage_graphs.erase(b->stage_graphs.begin() + g);
        b->stage_graphs.push_back(hit);
        for (int i = 0; i < b->count; ++i)  // what the captured stage did on the host
          states[i].t += stage_time_advance(rk_stage, dt);
        return launch(hit.exec);
      }
    }
  }
  // the stage advances every instance's state: no tuning runs on the caller's
  // data; the fork width is the Poisson batch's, else min(8, count)
  const int K = b->branches > 0 ? b->branches : std::min(8, b->count);
  cudaGraphExec_t exec = nullptr;
  {
    int rc = capture_stage(b, K, states, markers, rk_stage, dt, nu, st, &exec);
    if (rc) return rc;
  }
  int rc = launch(exec);
  if (!still) {
    IBM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaGraphExecDestroy(exec);
    return rc;
  }
  if (b->stage_graphs.size() >= 6) {
    cudaGraphExecDestroy(b->stage_graphs.front().exec);
    b->stage_graphs.erase(b->stage_graphs.begin());
  }
  b->stage_graphs.push_back({key, exec});
  return rc;
}

}  // extern "C"
