// plan.cu -- plan creation, the direct solve pipeline and the exported
// Poisson / Helmholtz entry points of libibm.
//
// Solve pipeline for one right-hand side (Sec. 2.3.3, doubly periodic
// branch: S1.1 + S1.2 for Helmholtz, S2.1 + S2.2 for Poisson):
//   1. forward real FFT along x and complex FFT along z of every y-plane;
//   2. one tridiagonal solve along y per Fourier pencil (pencil.cu);
//   3. inverse transforms, scaled by 1/(nx nz).
// FP32 plans then apply `refine` steps of iterative refinement: residual
// r = b - A x in float-float arithmetic (stencil.cu), correction solve of
// A d = r with the same pipeline, x += d fused into the inverse transform.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "plan.h"
#include "tma.cuh"

namespace ibm {

static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(IBM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return set_error(IBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool pdl_enabled() {
  static const bool on = !(getenv("IBM_PDL") && atoi(getenv("IBM_PDL")) == 0);
  return on;
}

TransformGeom geom_of(const ibm_plan_s *p) {
  TransformGeom g;
  g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
  g.nb = 1;
  g.use_plane = p->use_plane;
  g.err = p->derr;
  g.zrhs = nullptr;
  g.zsol = nullptr;
  g.dft_fwd = p->dftf;
  g.dft_inv = p->dfti;
  return g;
}

template <typename T>
static int upload_tables(ibm_plan_s *p) {
  const int nx = p->nx, nz = p->nz, P = p->P;
  std::vector<cplx<T>> twx(nx), twz(nz);
  for (int m = 0; m < nx; ++m) {
    const double a = 2.0 * M_PI * (double)m / nx;
    twx[m] = mk<T>((T)std::cos(a), (T)-std::sin(a));
  }
  for (int m = 0; m < nz; ++m) {
    const double a = 2.0 * M_PI * (double)m / nz;
    twz[m] = mk<T>((T)std::cos(a), (T)-std::sin(a));
  }
  // modified wavenumbers kappa'^2 = (2/h^2)(1 - cos(kappa h)), Appendix A
  std::vector<T> lx(P), lz(nz);
  for (int k = 0; k < P; ++k)
    lx[k] = (T)(2.0 / (p->h[0] * p->h[0]) * (1.0 - std::cos(2.0 * M_PI * k / nx)));
  for (int k = 0; k < nz; ++k)
    lz[k] = (T)(2.0 / (p->h[2] * p->h[2]) * (1.0 - std::cos(2.0 * M_PI * k / nz)));
  IBM_CUDA_TRY(cudaMemcpy(p->twx, twx.data(), sizeof(cplx<T>) * nx, cudaMemcpyHostToDevice));
  IBM_CUDA_TRY(cudaMemcpy(p->twz, twz.data(), sizeof(cplx<T>) * nz, cudaMemcpyHostToDevice));
  IBM_CUDA_TRY(cudaMemcpy(p->lamx, lx.data(), sizeof(T) * P, cudaMemcpyHostToDevice));
  IBM_CUDA_TRY(cudaMemcpy(p->lamz, lz.data(), sizeof(T) * nz, cudaMemcpyHostToDevice));
  if (p->bc == IBM_BC_TRIPLY_PERIODIC) {
    const int ny = p->ny;
    std::vector<cplx<T>> twy(ny);
    std::vector<T> ly(ny);
    for (int m = 0; m < ny; ++m) {
      const double a = 2.0 * M_PI * (double)m / ny;
      twy[m] = mk<T>((T)std::cos(a), (T)-std::sin(a));
      ly[m] = (T)(2.0 / (p->h[1] * p->h[1]) * (1.0 - std::cos(a)));
    }
    IBM_CUDA_TRY(cudaMemcpy(p->twy, twy.data(), sizeof(cplx<T>) * ny, cudaMemcpyHostToDevice));
    IBM_CUDA_TRY(cudaMemcpy(p->lamy, ly.data(), sizeof(T) * ny, cudaMemcpyHostToDevice));
  }
  return IBM_OK;
}

ProfScope::ProfScope(ibm_plan_s *plan, int k, cudaStream_t s, int n) : p(plan), kind(k), launches(n), st(s) {
  if (!p || !p->prof_on) return;
  if (p->evpool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p->evpool.push_back(e);
  }
  a = p->evpool.back();
  p->evpool.pop_back();
  cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b;
  if (p->evpool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) { p->evpool.push_back(a); return; }
  } else {
    b = p->evpool.back();
    p->evpool.pop_back();
  }
  cudaEventRecord(b, st);
  p->prof.push_back({kind, launches, a, b});
}

void InfoTrace::read(double *phase_ms) {
  for (int k = 0; k < IBM_K_COUNT; ++k) phase_ms[k] = 0.0;
  for (size_t i = mark; i < p->prof.size(); ++i) {
    const auto &r = p->prof[i];
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < IBM_K_COUNT)
      phase_ms[r.kind] += t;
  }
  if (!was_on) {  // the caller is not tracing: the call's records go back to the pool
    for (size_t i = mark; i < p->prof.size(); ++i) {
      p->evpool.push_back(p->prof[i].a);
      p->evpool.push_back(p->prof[i].b);
    }
    p->prof.resize(mark);
  }
}

int plan_status(ibm_plan_s *p, cudaStream_t st) {
  int w[2] = {0, 0};
  IBM_CUDA_TRY(cudaMemcpyAsync(w, p->derr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  IBM_CUDA_TRY(cudaStreamSynchronize(st));
  if (!w[0]) return IBM_OK;
  IBM_CUDA_TRY(cudaMemsetAsync(p->derr, 0, 2 * sizeof(int), st));
  if (w[0] & (kErrTimeout | kErrAlign))
    return set_error(IBM_ERR_TIMEOUT, "a kernel of this plan gave up a bounded wait (error word %d)%s", w[0],
                     (w[0] & kErrWall) ? "; markers were also rejected by the wall rule" : "");
  return set_error(IBM_ERR_ARG,
                   "%d marker(s) closer to a wall than the delta kernel's half-width (1.5 hy, 2 hy for the "
                   "4-point kernel) were rejected: neither interpolated nor spread",
                   w[1]);
}

static void plan_free(ibm_plan_s *p) {
  if (!p) return;
  for (auto &r : p->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : p->evpool) cudaEventDestroy(e);
  void *bufs[] = {p->S, p->Sx[0], p->Sx[1], p->work, p->bsave, p->sub[0], p->sub[1], p->sub[2], p->sub[3], p->twy, p->lamy,
                  p->twx, p->twz, p->lamx, p->lamz, p->dsc, p->mkbuf, p->derr, p->zbuf, p->gbuf, p->dftf, p->dfti};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (p->hsc) cudaFreeHost(p->hsc);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

static int dalloc(ibm_plan_s *p, void **ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_error(e, "cudaMalloc");
  }
  p->bytes += bytes;
  return IBM_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
bool default_use_slab(int precision, int bc, int nx, int ny, int nz) {
  // read per plan (A/B timing, tests): IBM_SLAB=0 never, IBM_SLAB=1 wherever the shape is supported, unset
  // the measured default: 256 x 256 slabs (GB300, refined 256^3 solve 0.317 against 0.332 ms split; at
  // 128^3 the split passes win, 0.055 against 0.064 ms)
  const char *env = getenv("IBM_SLAB");
  if (precision != IBM_FP32_REFINED || bc != IBM_BC_PXZ_WALL_Y || !slab_supported(nx, ny, nz)) return false;
  if (env) return atoi(env) != 0;
  return ny == 256 && nz == 256;
}

// The fused slab path: three passes, each reading and writing the field once.
static int solve_once_slab(ibm_plan_s *p, const PencilParams &pp, const float *in, float *out, const float *addend,
                           double *mean_out, cudaStream_t st, int first_phase = 0) {
  float2 *S = static_cast<float2 *>(p->S);
  const float2 *twx = static_cast<const float2 *>(p->twx), *twz = static_cast<const float2 *>(p->twz);
  const float *lamx = static_cast<const float *>(p->lamx), *lamz = static_cast<const float *>(p->lamz);
  const float scale = (float)(1.0 / ((double)p->nx * p->nz));
  static const int kinds[3] = {IBM_K_FORWARD, IBM_K_PENCIL, IBM_K_INVERSE};
  for (int phase = first_phase; phase < 3; ++phase) {
    ProfScope ps(p, kinds[phase], st);
    IBM_CUDA_TRY(launch_slab_solve(pp, p->nx, in, S, out, addend, twx, twz, lamx, lamz, mean_out, scale, st, phase));
  }
  return IBM_OK;
}

// FP32 single-field solves of the plan's slab kinds take the slab path.
static bool slab_applies(const ibm_plan_s *p, const PencilParams &pp) {
  return p->use_slab && pp.j0 == 0 && pp.nb == 1 && !pp.periodic;
}

template <typename T>
static int solve_once(ibm_plan_s *p, const PencilParams &pp, const T *in, T *out, const T *addend,
                      double *mean_out, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (slab_applies(p, pp)) return solve_once_slab(p, pp, in, out, addend, mean_out, st);
  }
  TransformGeom gf = geom_of(p), gi = geom_of(p);
  if (pp.zero_mode) {
    gf.zrhs = p->zbuf;                               // plane sums of b (FP64)
    if (!pp.periodic) gi.zsol = p->zbuf + p->ny;     // the wall branch's FP64 zero pencil
  }
  const TransformGeom &g = gf;
  cplx<T> *S = static_cast<cplx<T> *>(p->S);
  const cplx<T> *twx = static_cast<const cplx<T> *>(p->twx);
  const cplx<T> *twz = static_cast<const cplx<T> *>(p->twz);
  const int nl = transform_launches<T>(g);
  {
    ProfScope ps(p, IBM_K_FORWARD, st, nl);
    IBM_CUDA_TRY(launch_forward<T>(gf, ptr3(in), ptr3(S), twx, twz, (T)1, st));
  }
  {
    ProfScope ps(p, IBM_K_PENCIL, st);
    IBM_CUDA_TRY(launch_pencil<T>(pp, ptr3(S), static_cast<const T *>(p->lamx), static_cast<const T *>(p->lamz),
                                  mean_out, st));
  }
  {
    ProfScope ps(p, IBM_K_INVERSE, st, nl);
    IBM_CUDA_TRY(launch_inverse<T>(gi, ptr3(S), ptr3(out), ptr3(addend), twx, twz,
                                   (T)(1.0 / ((double)p->nx * p->nz)), st));
  }
  return IBM_OK;
}

static PencilParams pencil_params(const ibm_plan_s *p, int kind, double c, int field_bc) {
  PencilParams pp;
  std::memset(&pp, 0, sizeof pp);
  pp.ny = p->ny; pp.nz = p->nz; pp.P = p->P;
  const double hy = p->h[1];
  if (kind == 0) {
    pp.a = 1.0 / (hy * hy);
    pp.g_add = 0.0; pp.g_mul = 1.0;
    pp.beta_s = pp.beta_e = 0;
    pp.j0 = 0; pp.neg_rhs = 1; pp.zero_mode = 1;
  } else {
    pp.a = c / (hy * hy);
    pp.g_add = 1.0; pp.g_mul = c;
    const int beta = field_bc == IBM_FIELD_CELL_NEUMANN ? 0 : field_bc == IBM_FIELD_CELL_DIRICHLET ? 2 : 1;
    pp.beta_s = pp.beta_e = beta;
    pp.j0 = field_bc == IBM_FIELD_FACE_DIRICHLET ? 1 : 0;
    pp.neg_rhs = 0; pp.zero_mode = 0;
  }
  pp.hy2 = hy * hy;
  pp.inv_nxnz = 1.0 / ((double)p->nx * p->nz);
  pp.err = p->derr;
  pp.mode = p->pencil_mode;
  pp.zrhs = p->zbuf;
  pp.zsol = p->zbuf + p->ny;
  pp.inv_ny = 1.0 / p->ny;
  pp.nb = 1;
  if (p->bc == IBM_BC_TRIPLY_PERIODIC) {
    pp.periodic = 1;
    pp.twy = p->twy;
    pp.lamy = p->lamy;
    pp.beta_s = pp.beta_e = pp.j0 = 0;
  }
  return pp;
}

static StencilCoef stencil_coef(const ibm_plan_s *p, int kind, double c, int field_bc) {
  StencilCoef sc;
  sc.cx = 1.0 / (p->h[0] * p->h[0]);
  sc.cy = 1.0 / (p->h[1] * p->h[1]);
  sc.cz = 1.0 / (p->h[2] * p->h[2]);
  if (kind == 0) { sc.sigma = 0.0; sc.tau = 1.0; sc.bc = p->bc == IBM_BC_TRIPLY_PERIODIC ? IBM_FIELD_PERIODIC : 0; }
  else { sc.sigma = 1.0; sc.tau = -c; sc.bc = field_bc; }
  return sc;
}

template <typename T>
static int plan_solve_t(ibm_plan_s *p, int kind, double c, int field_bc, const T *in, T *out, const T *addend,
                        cudaStream_t st, ibm_info *info) {
  const PencilParams pp = pencil_params(p, kind, c, field_bc);
  const StencilCoef sc = stencil_coef(p, kind, c, field_bc);
  const int iters = (p->precision == IBM_FP32_REFINED && addend == nullptr) ? p->refine : 0;
  const bool need_b = iters > 0 || info;
  const T *b = in;
  if (need_b && (const void *)in == (const void *)out) {
    IBM_CUDA_TRY(cudaMemcpyAsync(p->bsave, in, p->npts * sizeof(T), cudaMemcpyDeviceToDevice, st));
    b = static_cast<const T *>(p->bsave);
  }
  InfoTrace trace(p, info != nullptr);
  if (info) {
    IBM_CUDA_TRY(cudaMemsetAsync(p->dsc, 0, 8 * sizeof(double), st));
    IBM_CUDA_TRY(cudaEventRecord(p->ev0, st));
  }
  int rc = solve_once<T>(p, pp, b, out, addend, kind == 0 ? p->dsc : nullptr, st);
  if (rc) return rc;
  T *r = static_cast<T *>(p->work);
  for (int it = 0; it < iters; ++it) {
    if constexpr (sizeof(T) == 4) {
      if (slab_applies(p, pp) && slab_residual_fused(p->nx, p->nz)) {  // r straight into the correction's x rows
        {
          ProfScope ps(p, IBM_K_RESIDUAL, st);
          IBM_CUDA_TRY(launch_slab_residual_forward(sc, p->nx, p->ny, p->nz, b, out, static_cast<float2 *>(p->S),
                                                    static_cast<const float2 *>(p->twx),
                                                    kind == 0 ? p->dsc : nullptr, nullptr, p->derr, st));
        }
        rc = solve_once_slab(p, pp, nullptr, out, out, nullptr, st, 1);
        if (rc) return rc;
        continue;
      }
    }
    {
      ProfScope ps(p, IBM_K_RESIDUAL, st);
      IBM_CUDA_TRY(launch_residual<T>(p->nx, p->ny, p->nz, sc, b, out, r, kind == 0 ? p->dsc : nullptr, nullptr,
                                      st));
    }
    rc = solve_once<T>(p, pp, r, out, out, nullptr, st);
    if (rc) return rc;
  }
  if (info) {
    IBM_CUDA_TRY(cudaEventRecord(p->ev1, st));
    // relative residual of the returned x (only meaningful without addend)
    IBM_CUDA_TRY(launch_residual<T>(p->nx, p->ny, p->nz, sc, b, out, r, kind == 0 ? p->dsc : nullptr, p->dsc + 4, st));
    IBM_CUDA_TRY(cudaMemcpyAsync(p->hsc, p->dsc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    IBM_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    IBM_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    const double N = (double)p->npts;
    const double *h = p->hsc;
    const double rr = std::max(0.0, h[4] - h[6] * h[6] / N);
    const double bb = h[5];
    trace.read(info->phase_ms);
    if ((rc = plan_status(p, st))) return rc;
    info->rel_residual = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    info->removed_mean = kind == 0 ? h[0] : 0.0;
    info->div_max = 0.0;
    info->div_before = 0.0;
    info->t_ms = ms;
    info->refine_iters = iters;
  }
  return IBM_OK;
}

template <typename T>
static int solve_fields_t(ibm_plan_s *p, double c, int nb, const int *field_bc, const T *const *in, T *const *out,
                          const T *const *addend, cudaStream_t st) {
  TransformGeom g = geom_of(p);
  g.nb = nb;
  g.use_plane = p->use_plane_fields;
  PencilParams pp = pencil_params(p, 1, c, field_bc[0]);
  pp.nb = nb;
  for (int b = 1; b < nb; ++b) {
    const PencilParams q = pencil_params(p, 1, c, field_bc[b]);
    pp.fbc[b] = q.beta_s | (q.beta_e << 4) | (q.j0 << 8);
  }
  Ptr3<cplx<T> *> S{{static_cast<cplx<T> *>(p->S), static_cast<cplx<T> *>(p->Sx[0]),
                     static_cast<cplx<T> *>(p->Sx[1])}};
  Ptr3<const T *> in3{{in[0], nb > 1 ? in[1] : nullptr, nb > 2 ? in[2] : nullptr}};
  Ptr3<T *> out3{{out[0], nb > 1 ? out[1] : nullptr, nb > 2 ? out[2] : nullptr}};
  Ptr3<const T *> add3{{addend[0], nb > 1 ? addend[1] : nullptr, nb > 2 ? addend[2] : nullptr}};
  const cplx<T> *twx = static_cast<const cplx<T> *>(p->twx);
  const cplx<T> *twz = static_cast<const cplx<T> *>(p->twz);
  const int nl = transform_launches<T>(g);
  {
    ProfScope ps(p, IBM_K_FORWARD, st, nl);
    IBM_CUDA_TRY(launch_forward<T>(g, in3, S, twx, twz, (T)1, st));
  }
  {
    ProfScope ps(p, IBM_K_PENCIL, st);
    IBM_CUDA_TRY(launch_pencil<T>(pp, S, static_cast<const T *>(p->lamx), static_cast<const T *>(p->lamz), nullptr,
                                  st));
  }
  {
    ProfScope ps(p, IBM_K_INVERSE, st, nl);
    IBM_CUDA_TRY(launch_inverse<T>(g, S, out3, add3, twx, twz, (T)(1.0 / ((double)p->nx * p->nz)), st));
  }
  return IBM_OK;
}

int plan_solve_fields(ibm_plan_s *p, double c, int nb, const int *field_bc, const void *const *in, void *const *out,
                      const void *const *addend, cudaStream_t st) {
  if (nb < 1 || nb > kMaxFields) return set_error(IBM_ERR_ARG, "plan_solve_fields: %d fields", nb);
  for (int b = 0; b + 1 < nb; ++b) {
    if (!p->Sx[b]) {
      cudaError_t e = cudaMalloc(&p->Sx[b], p->nspec * 2 * p->esz);
      if (e != cudaSuccess) { p->Sx[b] = nullptr; return cuda_error(e, "field spectrum"); }
      p->bytes += p->nspec * 2 * p->esz;
    }
  }
  if (p->precision == IBM_FP64)
    return solve_fields_t<double>(p, c, nb, field_bc, reinterpret_cast<const double *const *>(in),
                                  reinterpret_cast<double *const *>(out),
                                  reinterpret_cast<const double *const *>(addend), st);
  return solve_fields_t<float>(p, c, nb, field_bc, reinterpret_cast<const float *const *>(in),
                               reinterpret_cast<float *const *>(out), reinterpret_cast<const float *const *>(addend),
                               st);
}

int plan_solve(ibm_plan_s *p, int kind, double c, int field_bc, const void *in, void *out, const void *addend,
               cudaStream_t st, ibm_info *info) {
  if (p->precision == IBM_FP64)
    return plan_solve_t<double>(p, kind, c, field_bc, static_cast<const double *>(in), static_cast<double *>(out),
                                static_cast<const double *>(addend), st, info);
  return plan_solve_t<float>(p, kind, c, field_bc, static_cast<const float *>(in), static_cast<float *>(out),
                             static_cast<const float *>(addend), st, info);
}

// A solve with non-homogeneous wall data: the data's share of the operator
// moves to the right-hand side (a copy in bsave), the homogeneous solve runs
// on it, and a face field's wall plane gets its value.  Operator
// A x = sigma x + tau L x (Poisson: L; Helmholtz: I - c L); the ghost rules
// with wall data g (Appendix B) add B(g) to L x on the rows next to a wall:
//   cell Neumann (g = dx/dy at the wall)      row 0: -g_lo / hy,    row ny-1: +g_hi / hy
//   cell Dirichlet (g = the wall value)       row 0: +2 g_lo / hy^2, row ny-1: +2 g_hi / hy^2
//   face Dirichlet (g = the wall face value)  row 1: +g_lo / hy^2,   row ny-1: +g_hi / hy^2
// so the right-hand side becomes b - tau B(g).
static int solve_bc(ibm_plan_s *p, int kind, double c, int field_bc, const void *rhs, void *out, const void *glo,
                    const void *ghi, cudaStream_t st, ibm_info *info) {
  const double hy = p->h[1];
  const double tau = kind == 0 ? 1.0 : -c;
  const int fb = kind == 0 ? IBM_FIELD_CELL_NEUMANN : field_bc;
  double blo, bhi;
  int jlo = 0, jhi = p->ny - 1;
  if (fb == IBM_FIELD_CELL_NEUMANN) { blo = -1.0 / hy; bhi = 1.0 / hy; }
  else if (fb == IBM_FIELD_CELL_DIRICHLET) { blo = bhi = 2.0 / (hy * hy); }
  else { blo = bhi = 1.0 / (hy * hy); jlo = 1; }
  IBM_CUDA_TRY(cudaMemcpyAsync(p->bsave, rhs, p->npts * p->esz, cudaMemcpyDeviceToDevice, st));
  if (p->precision == IBM_FP64)
    IBM_CUDA_TRY(launch_wall_rhs<double>(p->nx, p->nz, static_cast<double *>(p->bsave), jlo, jhi,
                                         static_cast<const double *>(glo), static_cast<const double *>(ghi),
                                         -tau * blo, -tau * bhi, st));
  else
    IBM_CUDA_TRY(launch_wall_rhs<float>(p->nx, p->nz, static_cast<float *>(p->bsave), jlo, jhi,
                                        static_cast<const float *>(glo), static_cast<const float *>(ghi),
                                        -tau * blo, -tau * bhi, st));
  const int rc = plan_solve(p, kind, c, field_bc, p->bsave, out, nullptr, st, info);
  if (rc) return rc;
  if (fb == IBM_FIELD_FACE_DIRICHLET && glo)
    IBM_CUDA_TRY(cudaMemcpyAsync(out, glo, (size_t)p->nx * p->nz * p->esz, cudaMemcpyDeviceToDevice, st));
  return IBM_OK;
}

}  // namespace ibm

using namespace ibm;

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------
extern "C" {

const char *ibm_last_error(void) { return g_last_error.c_str(); }
const char *ibm_version(void) { return "libibm 0.1 (sm_103a)"; }

int ibm_plan_create(int nx, int ny, int nz, int bc, const double h[3], int precision, int refine_iters,
                    ibm_plan *out) {
  if (!out) return set_error(IBM_ERR_ARG, "ibm_plan_create: out is NULL");
  *out = nullptr;
  if (bc != IBM_BC_PXZ_WALL_Y && bc != IBM_BC_TRIPLY_PERIODIC)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_plan_create: unsupported bc %d", bc);
  if (bc == IBM_BC_TRIPLY_PERIODIC && !transform_size_supported(ny))
    return set_error(IBM_ERR_ARG, "ibm_plan_create: periodic ny=%d must be 2^a 3^b (b<=1) in [8,512]", ny);
  if (!transform_size_supported(nx) || !transform_size_supported(nz))
    return set_error(IBM_ERR_ARG, "ibm_plan_create: nx=%d nz=%d must be 2^a 3^b (b<=1) in [8,512]", nx, nz);
  if (ny < 8 || ny > 512) return set_error(IBM_ERR_ARG, "ibm_plan_create: ny=%d outside [8,512]", ny);
  if (!h || !(h[0] > 0) || !(h[1] > 0) || !(h[2] > 0) || !std::isfinite(h[0]) || !std::isfinite(h[1]) ||
      !std::isfinite(h[2]))
    return set_error(IBM_ERR_ARG, "ibm_plan_create: spacings must be finite and positive");
  if (precision != IBM_FP64 && precision != IBM_FP32_REFINED)
    return set_error(IBM_ERR_ARG, "ibm_plan_create: precision %d", precision);
  if (refine_iters < 0 || refine_iters > 4)
    return set_error(IBM_ERR_ARG, "ibm_plan_create: refine_iters %d outside [0,4]", refine_iters);
  ibm_plan_s *p = new (std::nothrow) ibm_plan_s();
  if (!p) return set_error(IBM_ERR_OOM, "ibm_plan_create: host allocation");
  p->nx = nx; p->ny = ny; p->nz = nz; p->P = nx / 2 + 1;
  p->bc = bc;
  p->h[0] = h[0]; p->h[1] = h[1]; p->h[2] = h[2];
  p->precision = precision;
  p->refine = precision == IBM_FP64 ? 0 : refine_iters;
  p->delta = IBM_DELTA_ROMA3;
  // pencil solver: FP32 the segmented sweep where ny allows, else the
  // two-ended sweep (tile or streaming kernel by size); IBM_PENCIL_MODE=m forces 1
  // (warp-parallel block solve), 2 (tile), 3 (streaming) or 4 (segmented)
  // for A/B timing and tests; the tuner may pick any of them
  p->pencil_mode = 0;
  if (const char *pm = getenv("IBM_PENCIL_MODE")) {
    const int m = atoi(pm);
    if (m < 0 || m > 4) {
      delete p;
      return set_error(IBM_ERR_ARG, "ibm_plan_create: IBM_PENCIL_MODE=%d outside [0,4]", m);
    }
    p->pencil_mode = m;
  }
  // plane transforms: the default mode for the shape; IBM_PLANE_MODE=m forces
  // mode m (0 split passes, 1 one CTA per plane, 2/4/8 cluster, -1 tensor-core
  // DFT products) and fails the plan when the shape has no such mode (A/B
  // timing and tests)
  p->use_plane = precision == IBM_FP64 ? default_plane_mode<double>(nx, ny, nz) : default_plane_mode<float>(nx, ny, nz);
  p->use_slab = default_use_slab(precision, bc, nx, ny, nz) ? 1 : 0;
  // three-field solves: split passes (their small CTAs share the SMs
  // between fields); IBM_PLANE_MODE_FIELDS=m forces another mode
  p->use_plane_fields = 0;
  if (const char *pm = getenv("IBM_PLANE_MODE_FIELDS")) {
    int modes[8];
    const int n = precision == IBM_FP64 ? plane_modes<double>(nx, nz, modes) : plane_modes<float>(nx, nz, modes);
    const int want = atoi(pm);
    bool found = false;
    for (int i = 0; i < n; ++i) found |= modes[i] == want;
    if (!found) {
      delete p;
      return set_error(IBM_ERR_UNSUPPORTED, "ibm_plan_create: IBM_PLANE_MODE_FIELDS=%d not available for %dx%d planes",
                       want, nx, nz);
    }
    p->use_plane_fields = want;
  }
  if (const char *pm = getenv("IBM_PLANE_MODE")) {
    int modes[8];
    const int n = precision == IBM_FP64 ? plane_modes<double>(nx, nz, modes) : plane_modes<float>(nx, nz, modes);
    const int want = atoi(pm);
    bool found = false;
    for (int i = 0; i < n; ++i) found |= modes[i] == want;
    if (!found) {
      delete p;
      return set_error(IBM_ERR_UNSUPPORTED, "ibm_plan_create: IBM_PLANE_MODE=%d not available for %dx%d planes", want,
                       nx, nz);
    }
    p->use_plane = want;
  }
  p->esz = precision == IBM_FP64 ? 8 : 4;
  p->npts = (size_t)nx * ny * nz;
  p->nspec = (size_t)ny * nz * p->P;
  int rc = IBM_OK;
  if ((rc = dalloc(p, &p->S, p->nspec * 2 * p->esz)) ||
      (rc = dalloc(p, &p->work, p->npts * p->esz)) ||
      (rc = dalloc(p, &p->bsave, p->npts * p->esz)) ||
      (rc = dalloc(p, &p->twx, (size_t)nx * 2 * p->esz)) ||
      (rc = dalloc(p, &p->twz, (size_t)nz * 2 * p->esz)) ||
      (rc = dalloc(p, &p->lamx, (size_t)p->P * p->esz)) ||
      (rc = dalloc(p, &p->lamz, (size_t)nz * p->esz)) ||
      (rc = dalloc(p, (void **)&p->dsc, 16 * sizeof(double))) ||
      (rc = dalloc(p, (void **)&p->derr, 16)) ||
      (rc = dalloc(p, (void **)&p->zbuf, 2 * (size_t)ny * sizeof(double))) ||
      (bc == IBM_BC_TRIPLY_PERIODIC && ((rc = dalloc(p, &p->twy, (size_t)ny * 2 * p->esz)) ||
                                        (rc = dalloc(p, &p->lamy, (size_t)ny * p->esz))))) {
    plan_free(p);
    return rc;
  }
  cudaError_t e = cudaMallocHost((void **)&p->hsc, 16 * sizeof(double));
  if (e != cudaSuccess) { plan_free(p); return cuda_error(e, "cudaMallocHost"); }
  if ((e = cudaEventCreate(&p->ev0)) != cudaSuccess || (e = cudaEventCreate(&p->ev1)) != cudaSuccess) {
    plan_free(p);
    return cuda_error(e, "cudaEventCreate");
  }
  if ((e = cudaMemset(p->derr, 0, 16)) != cudaSuccess) { plan_free(p); return cuda_error(e, "cudaMemset"); }
  rc = precision == IBM_FP64 ? upload_tables<double>(p) : upload_tables<float>(p);
  if (rc) { plan_free(p); return rc; }
  if (precision == IBM_FP32_REFINED && dft_tc_supported(nx, nz)) {
    size_t tb = 0;
    if ((e = dft_tc_upload(nx, nz, &p->dftf, &p->dfti, &tb)) != cudaSuccess) {
      plan_free(p);
      return cuda_error(e, "DFT tables");
    }
    p->bytes += tb;
  }
  *out = p;
  return IBM_OK;
}

int ibm_plan_destroy(ibm_plan plan) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_destroy: NULL plan");
  cudaDeviceSynchronize();
  plan_free(plan);
  return IBM_OK;
}

int ibm_plan_set_delta(ibm_plan plan, int kernel) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_set_delta: NULL plan");
  if (kernel != IBM_DELTA_ROMA3 && kernel != IBM_DELTA_PESKIN4)
    return set_error(IBM_ERR_ARG, "ibm_plan_set_delta: kernel %d", kernel);
  plan->delta = kernel;
  return IBM_OK;
}

int ibm_plan_set_spread(ibm_plan plan, int mode) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_set_spread: NULL plan");
  if (mode != IBM_SPREAD_ATOMIC && mode != IBM_SPREAD_GATHER && mode != IBM_SPREAD_ATOMIC_DIRECT)
    return set_error(IBM_ERR_ARG, "ibm_plan_set_spread: mode %d", mode);
  plan->spread = mode;
  return IBM_OK;
}

size_t ibm_plan_workspace_bytes(ibm_plan plan) { return plan ? plan->bytes : 0; }

int ibm_plan_check(ibm_plan plan) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_check: NULL plan");
  IBM_CUDA_TRY(cudaDeviceSynchronize());
  return plan_status(plan, 0);
}

int ibm_plan_profile(ibm_plan plan, int enable) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_profile: NULL plan");
  plan->prof_on = enable ? 1 : 0;
  return IBM_OK;
}

int ibm_plan_profile_read(ibm_plan plan, int max_kinds, double *ms, int *launches) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_plan_profile_read: NULL plan");
  IBM_CUDA_TRY(cudaDeviceSynchronize());
  double acc[IBM_K_COUNT] = {0};
  int cnt[IBM_K_COUNT] = {0};
  for (auto &r : plan->prof) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < IBM_K_COUNT) {
      acc[r.kind] += t;
      cnt[r.kind] += r.launches;
    }
    plan->evpool.push_back(r.a);
    plan->evpool.push_back(r.b);
  }
  plan->prof.clear();
  for (int k = 0; k < max_kinds && k < IBM_K_COUNT; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = cnt[k];
  }
  return IBM_K_COUNT;
}

int ibm_poisson_solve(ibm_plan plan, const void *rhs, void *phi, void *stream, ibm_info *info) {
  if (!plan || !rhs || !phi) return set_error(IBM_ERR_ARG, "ibm_poisson_solve: NULL argument");
  if (!aligned_to(rhs, 16) || !aligned_to(phi, 16))
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve: field pointers must be 16-byte aligned");
  return plan_solve(plan, 0, 0.0, 0, rhs, phi, nullptr, (cudaStream_t)stream, info);
}

int ibm_helmholtz_solve(ibm_plan plan, double c, int field_bc, const void *rhs, void *u, void *stream,
                        ibm_info *info) {
  if (!plan || !rhs || !u) return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c)) return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve: c must be > 0");
  if (plan->bc == IBM_BC_TRIPLY_PERIODIC ? field_bc != IBM_FIELD_PERIODIC
                                          : (field_bc < IBM_FIELD_CELL_NEUMANN || field_bc > IBM_FIELD_FACE_DIRICHLET))
    return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve: field_bc %d for this plan's bc", field_bc);
  if (!aligned_to(rhs, 16) || !aligned_to(u, 16))
    return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve: field pointers must be 16-byte aligned");
  return plan_solve(plan, 1, c, field_bc, rhs, u, nullptr, (cudaStream_t)stream, info);
}

int ibm_poisson_solve_bc(ibm_plan plan, const void *rhs, void *phi, const void *q_lo, const void *q_hi, void *stream,
                         ibm_info *info) {
  if (!plan || !rhs || !phi) return set_error(IBM_ERR_ARG, "ibm_poisson_solve_bc: NULL argument");
  if (plan->bc == IBM_BC_TRIPLY_PERIODIC)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_poisson_solve_bc: the triply periodic branch has no walls");
  if (!aligned_to(rhs, 16) || !aligned_to(phi, 16) || !aligned_to(q_lo, 16) || !aligned_to(q_hi, 16))
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_bc: field pointers must be 16-byte aligned");
  return solve_bc(plan, 0, 0.0, 0, rhs, phi, q_lo, q_hi, (cudaStream_t)stream, info);
}

int ibm_helmholtz_solve_bc(ibm_plan plan, double c, int field_bc, const void *rhs, void *u, const void *g_lo,
                           const void *g_hi, void *stream, ibm_info *info) {
  if (!plan || !rhs || !u) return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve_bc: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c)) return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve_bc: c must be > 0");
  if (plan->bc == IBM_BC_TRIPLY_PERIODIC)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_helmholtz_solve_bc: the triply periodic branch has no walls");
  if (field_bc < IBM_FIELD_CELL_NEUMANN || field_bc > IBM_FIELD_FACE_DIRICHLET)
    return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve_bc: field_bc %d", field_bc);
  if (!aligned_to(rhs, 16) || !aligned_to(u, 16) || !aligned_to(g_lo, 16) || !aligned_to(g_hi, 16))
    return set_error(IBM_ERR_ARG, "ibm_helmholtz_solve_bc: field pointers must be 16-byte aligned");
  return solve_bc(plan, 1, c, field_bc, rhs, u, g_lo, g_hi, (cudaStream_t)stream, info);
}

}  // extern "C"
