// server.cu -- continuous-batching request server (ibm_server_*).
//
// Requests (Poisson, Helmholtz or one RK stage) arrive with FP64 host
// buffers (IBM_DATA_HOST_FP64) or with device buffers in the plan precision
// (IBM_DATA_DEVICE, solved in place of the caller's output with no staging).
// A scheduler thread
//   * admits queued requests in arrival order whenever a stream slot is free
//     and the request's device memory fits the HBM budget: resident plans are
//     reused per (shape, precision, refinement); idle ones are evicted least
//     recently used first when memory is short; a request that cannot fit
//     even in an empty server fails with IBM_ERR_OOM;
//   * stages each admitted request through the slot's pinned buffer, copies
//     it to the device, converts FP64 -> plan precision on the device, runs
//     the solve on the slot's stream, converts back and copies out, with
//     events around the device work;
//   * hands each admitted request to its slot's worker thread, which stages
//     it, launches it, waits for its stream and copies the result into the
//     caller's output buffer -- so host staging of different slots runs in
//     parallel.
// Each slot keeps grow-only pinned and device staging buffers, so steady
// state serving allocates nothing (a cudaFree would synchronise the device);
// large host copies into and out of them run on several threads.
// Requests on different slots run concurrently on the device while new ones
// keep being admitted.  ibm_poll / ibm_wait report completion.  The host-side
// fault hook IBM_FAULT_ADMIT=N makes the N-th admission fail (IBM_ERR_OOM) to
// exercise error paths without touching the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace ibm {

template <typename T>
__global__ void k_from_f64(const double *__restrict__ in, T *__restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}
template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// Host copy between a caller's buffer and a slot's pinned staging buffer.
// Copies of 16 MB and more are split over up to 4 threads: the largest
// requests (an RK stage at 128^3 carries 67 MB of FP64 fields each way)
// would otherwise spend milliseconds in one core's memcpy.  Measured on the
// GB300 host (2000 req/s sample): FP32 p99 10.8 -> 3.8 ms; 8 threads gave
// no more (the copy is then bound by host memory bandwidth).
static void stage_copy(void *dst, const void *src, size_t bytes) {
  constexpr size_t kChunk = 8u << 20;
  const int nt = (int)std::min<size_t>(4, bytes / kChunk);
  if (nt < 2) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t part = (bytes / nt + 63) / 64 * 64;
  std::vector<std::thread> th;
  size_t done_from = bytes;  // parts from here on are copied by this thread (a helper could not start)
  for (int t = 1; t < nt; ++t) {
    const size_t off = part * t;
    if (off >= bytes) break;
    try {
      th.emplace_back([=] {
        std::memcpy(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off,
                    std::min(part, bytes - off));
      });
    } catch (...) {
      done_from = off;
      break;
    }
  }
  std::memcpy(dst, src, std::min(part, bytes));
  if (done_from < bytes)
    std::memcpy(static_cast<char *>(dst) + done_from, static_cast<const char *>(src) + done_from, bytes - done_from);
  for (auto &x : th) x.join();
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct PlanKey {
  int nx, ny, nz, precision, refine;
  bool operator==(const PlanKey &o) const {
    return nx == o.nx && ny == o.ny && nz == o.nz && precision == o.precision && refine == o.refine;
  }
};

struct Resident {
  PlanKey key;
  ibm_plan_s *plan;
  bool busy;
  double last_use;
  size_t bytes;
};

struct Req {
  uint64_t ticket;
  ibm_request r;
  int status = IBM_PENDING;
  double t_submit = 0, t_admit = 0, t_done = 0;
  float device_ms = 0;
  double removed_mean = 0;
  int slot = -1;
  Resident *res = nullptr;
  void *dmem = nullptr;
  size_t dbytes = 0;
  size_t out_bytes = 0;
};

struct Slot {
  std::thread worker;      // stages, launches and retires this slot's requests
  std::condition_variable cv;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void *pinned = nullptr;  // host staging, grow-only
  size_t pinned_bytes = 0;
  void *dev = nullptr;     // device staging and fields, grow-only (no cudaFree between requests: it
  size_t dev_bytes = 0;    // would synchronise the device and serialise the slots)
  Req *req = nullptr;
};

}  // namespace ibm

using namespace ibm;

struct ibm_server_s {
  size_t budget = 0, used = 0;
  int max_queue = 0;
  std::unique_ptr<Slot[]> slots;  // fixed array: slots hold threads and condition variables
  int nslots = 0;
  std::vector<Resident *> plans;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<Req *> queue;
  std::unordered_map<uint64_t, Req *> reqs;
  uint64_t next_ticket = 1;
  std::thread th;
  bool stop = false;
  long admissions = 0;
  long fault_admit = -1;
  int device = 0;
};

namespace ibm {

static size_t npts_of(const ibm_request &r) { return (size_t)r.nx * r.ny * r.nz; }
static size_t esz_of(const ibm_request &r) { return r.precision == IBM_FP64 ? 8 : 4; }
static int nfields_of(const ibm_request &r) { return r.kind == IBM_REQ_SUBSTEP ? 4 : 1; }

// Device bytes a request needs besides its plan: FP64 staging of the
// largest buffer, plan-precision fields and markers (device data: the stage's
// advection fields and marker outputs only).
static size_t io_bytes(const ibm_request &r) {
  const size_t n = npts_of(r), e = esz_of(r);
  if (r.data == IBM_DATA_DEVICE) {
    if (r.kind != IBM_REQ_SUBSTEP) return 4096;
    const size_t m = (size_t)std::max(0, r.n_markers);
    return 3 * n * e + m * e * 9 + 3 * 4096;
  }
  if (r.kind == IBM_REQ_SUBSTEP) {
    const size_t m = (size_t)std::max(0, r.n_markers);
    return 4 * n * 8 + 7 * n * e + m * (3 * 8 + 8) + m * e * (3 + 1 + 3 + 3 + 3) + 4096;
  }
  return n * 8 + 2 * n * e + 4096;
}
// Estimated bytes of a plan for this request's shape (substep plans also
// hold four stage fields).
static size_t plan_bytes_estimate(const ibm_request &r) {
  const size_t n = npts_of(r), e = esz_of(r);
  const size_t spec = (size_t)r.ny * r.nz * (r.nx / 2 + 1) * 2 * e;
  size_t b = spec + 2 * n * e + 65536;
  if (r.kind == IBM_REQ_SUBSTEP) b += 4 * n * e + (size_t)std::max(0, r.n_markers) * 3 * e;
  return b;
}

// The request's device memory is its slot's buffer; nothing to free here.
static void free_req_device(ibm_server_s *, Req *q) {
  q->dmem = nullptr;
  q->dbytes = 0;
}

static void evict_idle_locked(ibm_server_s *s, size_t need) {
  while (s->used + need > s->budget) {
    Resident *victim = nullptr;
    for (auto *r : s->plans)
      if (!r->busy && (!victim || r->last_use < victim->last_use)) victim = r;
    if (!victim) return;
    ibm_plan_destroy(victim->plan);
    s->used -= victim->bytes;
    s->plans.erase(std::find(s->plans.begin(), s->plans.end(), victim));
    delete victim;
  }
}

template <typename T> static cudaError_t convert_in(const double *src, T *dst, size_t n, cudaStream_t st) {
  k_from_f64<T><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template <typename T> static cudaError_t convert_out(const T *src, double *dst, size_t n, cudaStream_t st) {
  k_to_f64<T><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// Device data (IBM_DATA_DEVICE): the solve reads the caller's `in` and
// writes its `out`; a stage copies `in` to `out` and advances it in place,
// with the advection fields and marker outputs in the slot's buffer.
static int launch_device(Req *q, Slot &sl) {
  const ibm_request &r = q->r;
  const size_t n = npts_of(r), e = esz_of(r);
  const size_t nm = (size_t)std::max(0, r.n_markers);
  cudaStream_t st = sl.st;
  ibm_plan_s *p = q->res->plan;
  q->out_bytes = 0;
  IBM_CUDA_TRY(cudaEventRecord(sl.e0, st));
  int rc = IBM_OK;
  if (r.kind == IBM_REQ_POISSON || r.kind == IBM_REQ_HELMHOLTZ) {
    rc = r.kind == IBM_REQ_POISSON ? plan_solve(p, 0, 0.0, 0, r.in, r.out, nullptr, st, nullptr)
                                   : plan_solve(p, 1, r.c, r.field_bc, r.in, r.out, nullptr, st, nullptr);
    if (rc) return rc;
  } else {
    unsigned char *dp = static_cast<unsigned char *>(sl.dev);
    auto take = [&](size_t bytes) {
      unsigned char *x = dp;
      dp += (bytes + 255) / 256 * 256;
      return (void *)x;
    };
    IBM_CUDA_TRY(cudaMemcpyAsync(r.out, r.in, 4 * n * e, cudaMemcpyDeviceToDevice, st));
    void *N[3];
    for (int c = 0; c < 3; ++c) {
      N[c] = take(n * e);
      IBM_CUDA_TRY(cudaMemsetAsync(N[c], 0, n * e, st));
    }
    void *X = take(nm * 3 * e), *Ud = take(nm * 3 * e), *F = take(nm * 3 * e);
    unsigned char *f = static_cast<unsigned char *>(r.out);
    ibm_state stt{f, f + n * e, f + 2 * n * e, f + 3 * n * e, N[0], N[1], N[2], 0.0};
    ibm_markers mk{};
    mk.n = (int)nm;
    mk.X0 = r.X0;
    mk.dV = r.dV;
    mk.X = X;
    mk.Ud = Ud;
    mk.F = F;
    mk.motion = r.motion;
    for (int k = 0; k < 4; ++k) mk.params[k] = r.params[k];
    rc = ibm_substep(p, &stt, r.rk_stage, r.dt, r.nu, nm ? &mk : nullptr, st, nullptr);
    if (rc) return rc;
  }
  IBM_CUDA_TRY(cudaEventRecord(sl.e1, st));
  return IBM_OK;
}

// Stages and launches the device work of an admitted request on its slot
// (worker thread, server lock not held); returns an IBM_* code.
static int launch(ibm_server_s *s, Req *q, Slot &sl) {
  const ibm_request &r = q->r;
  const size_t n = npts_of(r), e = esz_of(r);
  const int nf = nfields_of(r);
  const size_t nm = (size_t)std::max(0, r.n_markers);
  if (r.data == IBM_DATA_DEVICE) {
    q->dbytes = io_bytes(r);
    if (sl.dev_bytes < q->dbytes) {
      // admission already reserved the growth in s->used
      if (sl.dev) cudaFree(sl.dev);
      sl.dev = nullptr;
      cudaError_t e2 = cudaMalloc(&sl.dev, q->dbytes);
      if (e2 != cudaSuccess) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->used -= q->dbytes;
        sl.dev_bytes = 0;
        return cuda_error(e2, "server slot buffer");
      }
      sl.dev_bytes = q->dbytes;
    }
    q->dmem = sl.dev;
    return launch_device(q, sl);
  }
  const size_t in_host = nf * n * 8 + (r.kind == IBM_REQ_SUBSTEP ? nm * 4 * 8 : 0);
  // pinned staging for the slot
  if (sl.pinned_bytes < in_host) {
    if (sl.pinned) cudaFreeHost(sl.pinned);
    sl.pinned = nullptr;
    sl.pinned_bytes = 0;
    IBM_CUDA_TRY(cudaMallocHost(&sl.pinned, in_host));
    sl.pinned_bytes = in_host;
  }
  q->dbytes = io_bytes(r);
  if (sl.dev_bytes < q->dbytes) {
    // admission already reserved the growth in s->used
    if (sl.dev) cudaFree(sl.dev);
    sl.dev = nullptr;
    cudaError_t e = cudaMalloc(&sl.dev, q->dbytes);
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lock(s->mu);
      s->used -= q->dbytes;  // the old buffer and the reserved growth
      sl.dev_bytes = 0;
      return cuda_error(e, "server slot buffer");
    }
    sl.dev_bytes = q->dbytes;
  }
  q->dmem = sl.dev;
  unsigned char *d = static_cast<unsigned char *>(q->dmem);
  double *d64 = reinterpret_cast<double *>(d);  // FP64 staging of all fields (+ markers)
  unsigned char *dp = d + (nf * n * 8 + (r.kind == IBM_REQ_SUBSTEP ? nm * 4 * 8 : 0) + 255) / 256 * 256;
  auto take = [&](size_t bytes) {
    unsigned char *p = dp;
    dp += (bytes + 255) / 256 * 256;
    return (void *)p;
  };
  double *h = static_cast<double *>(sl.pinned);
  stage_copy(h, r.in, nf * n * 8);
  if (r.kind == IBM_REQ_SUBSTEP && nm) {
    std::memcpy(h + nf * n, r.X0, nm * 3 * 8);
    std::memcpy(h + nf * n + nm * 3, r.dV, nm * 8);
  }
  cudaStream_t st = sl.st;
  IBM_CUDA_TRY(cudaMemcpyAsync(d64, h, in_host, cudaMemcpyHostToDevice, st));
  IBM_CUDA_TRY(cudaEventRecord(sl.e0, st));
  ibm_plan_s *p = q->res->plan;
  const bool f64 = r.precision == IBM_FP64;
  auto conv_in = [&](const double *src, void *dst, size_t cnt) {
    return f64 ? convert_in<double>(src, (double *)dst, cnt, st) : convert_in<float>(src, (float *)dst, cnt, st);
  };
  auto conv_out = [&](const void *src, double *dst, size_t cnt) {
    return f64 ? convert_out<double>((const double *)src, dst, cnt, st)
               : convert_out<float>((const float *)src, dst, cnt, st);
  };
  int rc = IBM_OK;
  if (r.kind == IBM_REQ_POISSON || r.kind == IBM_REQ_HELMHOLTZ) {
    void *fin = take(n * e), *fout = take(n * e);
    IBM_CUDA_TRY(conv_in(d64, fin, n));
    rc = r.kind == IBM_REQ_POISSON ? plan_solve(p, 0, 0.0, 0, fin, fout, nullptr, st, nullptr)
                                   : plan_solve(p, 1, r.c, r.field_bc, fin, fout, nullptr, st, nullptr);
    if (rc) return rc;
    IBM_CUDA_TRY(conv_out(fout, d64, n));
  } else {
    void *f[4], *N[3];
    for (int c = 0; c < 4; ++c) {
      f[c] = take(n * e);
      IBM_CUDA_TRY(conv_in(d64 + c * n, f[c], n));
    }
    for (int c = 0; c < 3; ++c) {
      N[c] = take(n * e);
      IBM_CUDA_TRY(cudaMemsetAsync(N[c], 0, n * e, st));
    }
    void *X0 = take(nm * 3 * e), *dV = take(nm * e), *X = take(nm * 3 * e), *Ud = take(nm * 3 * e),
         *F = take(nm * 3 * e);
    if (nm) {
      IBM_CUDA_TRY(conv_in(d64 + 4 * n, X0, nm * 3));
      IBM_CUDA_TRY(conv_in(d64 + 4 * n + nm * 3, dV, nm));
    }
    ibm_state stt{f[0], f[1], f[2], f[3], N[0], N[1], N[2], 0.0};
    ibm_markers mk{};
    mk.n = (int)nm;
    mk.X0 = X0;
    mk.dV = dV;
    mk.X = X;
    mk.Ud = Ud;
    mk.F = F;
    mk.motion = r.motion;
    for (int k = 0; k < 4; ++k) mk.params[k] = r.params[k];
    rc = ibm_substep(p, &stt, r.rk_stage, r.dt, r.nu, nm ? &mk : nullptr, st, nullptr);
    if (rc) return rc;
    for (int c = 0; c < 4; ++c) IBM_CUDA_TRY(conv_out(f[c], d64 + c * n, n));
  }
  IBM_CUDA_TRY(cudaEventRecord(sl.e1, st));
  q->out_bytes = nf * n * 8;
  IBM_CUDA_TRY(cudaMemcpyAsync(sl.pinned, d64, q->out_bytes, cudaMemcpyDeviceToHost, st));
  return IBM_OK;
}

static bool admit_one_locked(ibm_server_s *s) {
  if (s->queue.empty()) return false;
  int slot = -1;
  for (int k = 0; k < s->nslots; ++k)
    if (!s->slots[k].req) { slot = k; break; }
  if (slot < 0) return false;
  Req *q = s->queue.front();
  const ibm_request &r = q->r;
  const PlanKey key{r.nx, r.ny, r.nz, r.precision, r.refine_iters};
  Resident *res = nullptr;
  for (auto *x : s->plans)
    if (!x->busy && x->key == key) { res = x; break; }
  const size_t io = io_bytes(r);
  const size_t grow = io > s->slots[slot].dev_bytes ? io - s->slots[slot].dev_bytes : 0;
  const size_t need = grow + (res ? 0 : plan_bytes_estimate(r));
  bool fail_oom = false;
  if (s->fault_admit >= 0 && s->admissions == s->fault_admit) fail_oom = true;
  if (!fail_oom && s->used + need > s->budget) {
    evict_idle_locked(s, need);
    if (s->used + need > s->budget) {
      bool busy = false;
      for (int k = 0; k < s->nslots; ++k) busy = busy || s->slots[k].req;
      if (busy) return false;  // wait for running requests to free memory
      fail_oom = true;         // cannot fit even in an empty server
    }
  }
  s->queue.pop_front();
  s->admissions++;
  q->t_admit = now_ms();
  auto fail = [&](int code) {
    q->status = code;
    q->t_done = now_ms();
    free_req_device(s, q);
    if (q->res) q->res->busy = false;
    s->cv_done.notify_all();
  };
  if (fail_oom) {
    set_error(IBM_ERR_OOM, "request %llu does not fit the server's HBM budget", (unsigned long long)q->ticket);
    fail(IBM_ERR_OOM);
    return true;
  }
  if (!res) {
    ibm_plan_s *p = nullptr;
    int rc = ibm_plan_create(r.nx, r.ny, r.nz, IBM_BC_PXZ_WALL_Y, r.h, r.precision, r.refine_iters, &p);
    if (rc) {
      fail(rc);
      return true;
    }
    res = new Resident{key, p, false, 0.0, plan_bytes_estimate(r)};
    s->plans.push_back(res);
    s->used += res->bytes;
  }
  res->busy = true;
  res->last_use = now_ms();
  q->res = res;
  q->slot = slot;
  Slot &sl = s->slots[slot];
  if (io > sl.dev_bytes) s->used += io - sl.dev_bytes;  // the worker grows the slot buffer
  sl.req = q;
  sl.cv.notify_one();
  return true;
}

// Worker of one slot: waits for an admitted request, stages it, runs it,
// waits for its stream, copies the result out and hands the slot back.
// Host staging copies of different slots run in parallel.
static void slot_worker(ibm_server_s *s, int k) {
  cudaSetDevice(s->device);
  Slot &sl = s->slots[k];
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    sl.cv.wait(lock, [&] { return s->stop || (sl.req && sl.req->status == IBM_PENDING && sl.req->slot == k); });
    if (!sl.req) return;  // stopping with nothing assigned
    Req *q = sl.req;
    lock.unlock();
    int rc = launch(s, q, sl);
    cudaError_t e = cudaStreamSynchronize(sl.st);
    if (rc == IBM_OK && e != cudaSuccess) rc = cuda_error(e, "server request");
    // a bounded wait that gave up, or markers rejected by the wall rule,
    // fail this request (the resident plan's word is cleared for the next)
    if (rc == IBM_OK) rc = plan_status(q->res->plan, sl.st);
    if (rc == IBM_OK) {
      if (q->r.data == IBM_DATA_HOST_FP64) stage_copy(q->r.out, sl.pinned, q->out_bytes);
      cudaEventElapsedTime(&q->device_ms, sl.e0, sl.e1);
    }
    lock.lock();
    q->status = rc;
    q->t_done = now_ms();
    free_req_device(s, q);
    q->res->busy = false;
    q->res->last_use = now_ms();
    sl.req = nullptr;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    if (s->stop) return;
  }
}

static void scheduler(ibm_server_s *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    bool progressed = false;
    while (admit_one_locked(s)) progressed = true;
    if (!progressed) s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
  }
}

static int validate_request(const ibm_request *r) {
  if (!r) return set_error(IBM_ERR_ARG, "ibm_submit: NULL request");
  if (r->kind < IBM_REQ_POISSON || r->kind > IBM_REQ_SUBSTEP) return set_error(IBM_ERR_ARG, "ibm_submit: kind");
  if (!transform_size_supported(r->nx) || !transform_size_supported(r->nz) || r->ny < 8 || r->ny > 512)
    return set_error(IBM_ERR_ARG, "ibm_submit: unsupported grid %dx%dx%d", r->nx, r->ny, r->nz);
  if (!(r->h[0] > 0 && r->h[1] > 0 && r->h[2] > 0)) return set_error(IBM_ERR_ARG, "ibm_submit: spacings");
  if (r->precision != IBM_FP64 && r->precision != IBM_FP32_REFINED)
    return set_error(IBM_ERR_ARG, "ibm_submit: precision");
  if (r->refine_iters < 0 || r->refine_iters > 4) return set_error(IBM_ERR_ARG, "ibm_submit: refine_iters");
  if (!r->in || !r->out) return set_error(IBM_ERR_ARG, "ibm_submit: NULL in/out");
  if (r->data != IBM_DATA_HOST_FP64 && r->data != IBM_DATA_DEVICE)
    return set_error(IBM_ERR_ARG, "ibm_submit: data %d", r->data);
  if (r->data == IBM_DATA_DEVICE) {
    if (r->in == r->out) return set_error(IBM_ERR_ARG, "ibm_submit: device in and out must be distinct");
    if (!aligned_to(r->in, 16) || !aligned_to(r->out, 16))
      return set_error(IBM_ERR_ARG, "ibm_submit: device fields must be 16-byte aligned");
  }
  if (r->kind == IBM_REQ_HELMHOLTZ && (!(r->c > 0) || r->field_bc < 0 || r->field_bc > 2))
    return set_error(IBM_ERR_ARG, "ibm_submit: Helmholtz c / field_bc");
  if (r->kind == IBM_REQ_SUBSTEP) {
    if (r->rk_stage < 1 || r->rk_stage > 3 || !(r->dt > 0) || !(r->nu > 0))
      return set_error(IBM_ERR_ARG, "ibm_submit: substep stage / dt / nu");
    if (r->n_markers < 0 || (r->n_markers > 0 && (!r->X0 || !r->dV)))
      return set_error(IBM_ERR_ARG, "ibm_submit: markers");
  }
  return IBM_OK;
}

}  // namespace ibm

extern "C" {

int ibm_server_create(size_t hbm_budget_bytes, int n_streams, int max_queue, ibm_server *out) {
  if (!out || hbm_budget_bytes == 0 || n_streams < 1 || n_streams > 64 || max_queue < 1)
    return set_error(IBM_ERR_ARG, "ibm_server_create: bad arguments");
  *out = nullptr;
  ibm_server_s *s = new (std::nothrow) ibm_server_s();
  if (!s) return set_error(IBM_ERR_OOM, "ibm_server_create: host allocation");
  s->budget = hbm_budget_bytes;
  s->max_queue = max_queue;
  cudaGetDevice(&s->device);
  if (const char *f = getenv("IBM_FAULT_ADMIT")) s->fault_admit = atol(f);
  s->slots.reset(new (std::nothrow) Slot[n_streams]);
  if (!s->slots) {
    delete s;
    return set_error(IBM_ERR_OOM, "ibm_server_create: host allocation");
  }
  s->nslots = n_streams;
  for (int k = 0; k < n_streams; ++k) {
    Slot &sl = s->slots[k];
    cudaError_t e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.e1);
    if (e != cudaSuccess) {
      ibm_server_destroy(s);
      return cuda_error(e, "ibm_server_create");
    }
  }
  for (int k = 0; k < n_streams; ++k) s->slots[k].worker = std::thread(slot_worker, s, k);
  s->th = std::thread(scheduler, s);
  *out = s;
  return IBM_OK;
}

int ibm_server_destroy(ibm_server s) {
  if (!s) return set_error(IBM_ERR_ARG, "ibm_server_destroy: NULL server");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (int k = 0; k < s->nslots; ++k) s->slots[k].cv.notify_all();
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  for (int k = 0; k < s->nslots; ++k)
    if (s->slots[k].worker.joinable()) s->slots[k].worker.join();
  for (int k = 0; k < s->nslots; ++k) {
    Slot &sl = s->slots[k];
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.e0) cudaEventDestroy(sl.e0);
    if (sl.e1) cudaEventDestroy(sl.e1);
    if (sl.pinned) cudaFreeHost(sl.pinned);
    if (sl.dev) cudaFree(sl.dev);
  }
  for (auto *r : s->plans) {
    ibm_plan_destroy(r->plan);
    delete r;
  }
  for (auto &kv : s->reqs) {
    free_req_device(s, kv.second);
    delete kv.second;
  }
  delete s;
  return IBM_OK;
}

int ibm_submit(ibm_server s, const ibm_request *req, uint64_t *ticket) {
  if (!s || !ticket) return set_error(IBM_ERR_ARG, "ibm_submit: NULL argument");
  int rc = validate_request(req);
  if (rc) return rc;
  Req *q = new (std::nothrow) Req();
  if (!q) return set_error(IBM_ERR_OOM, "ibm_submit: host allocation");
  q->r = *req;
  q->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if ((int)s->queue.size() >= s->max_queue) {
      delete q;
      return set_error(IBM_ERR_BUSY, "ibm_submit: queue full (%d)", s->max_queue);
    }
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->queue.push_back(q);
    *ticket = q->ticket;
  }
  s->cv_work.notify_one();
  return IBM_OK;
}

static int poll_locked(ibm_server_s *s, uint64_t ticket, ibm_result *out) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(IBM_ERR_ARG, "ibm_poll: unknown ticket %llu", (unsigned long long)ticket);
  Req *q = it->second;
  if (q->status == IBM_PENDING) {
    if (out) out->status = IBM_PENDING;
    return IBM_PENDING;
  }
  if (out) {
    out->status = q->status;
    out->queue_ms = q->t_admit - q->t_submit;
    out->device_ms = q->device_ms;
    out->total_ms = q->t_done - q->t_submit;
    out->removed_mean = q->removed_mean;
  }
  const int st = q->status;
  s->reqs.erase(it);
  delete q;
  return st;
}

int ibm_poll(ibm_server s, uint64_t ticket, ibm_result *out) {
  if (!s) return set_error(IBM_ERR_ARG, "ibm_poll: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  return poll_locked(s, ticket, out);
}

int ibm_wait(ibm_server s, uint64_t ticket, double timeout_s, ibm_result *out) {
  if (!s) return set_error(IBM_ERR_ARG, "ibm_wait: NULL server");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    int rc = poll_locked(s, ticket, out);
    if (rc != IBM_PENDING) return rc;
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
      rc = poll_locked(s, ticket, out);
      if (rc != IBM_PENDING) return rc;
      return set_error(IBM_ERR_TIMEOUT, "ibm_wait: ticket %llu not done after %.3f s", (unsigned long long)ticket,
                       timeout_s);
    }
  }
}

int ibm_cancel(ibm_server s, uint64_t ticket) {
  if (!s) return set_error(IBM_ERR_ARG, "ibm_cancel: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(IBM_ERR_ARG, "ibm_cancel: unknown ticket");
  auto qi = std::find(s->queue.begin(), s->queue.end(), it->second);
  if (qi == s->queue.end()) return set_error(IBM_ERR_BUSY, "ibm_cancel: request already admitted");
  s->queue.erase(qi);
  it->second->status = IBM_ERR_CANCELLED;
  it->second->t_admit = it->second->t_done = now_ms();
  s->cv_done.notify_all();
  return IBM_OK;
}

}  // extern "C"
