// noalloc.cu -- FP32 Poisson solve that allocates no device memory.
//
// Some callers cannot allocate GPU memory at solve time: code running under
// a memory pool or a device-memory budget owned by someone else (a host
// framework that hands out only the buffers it manages), code that must not
// call cudaMalloc because that call synchronises the device or may fail late
// in a long run, and code embedded where only pre-existing buffers may be
// touched.  For them ibm_poisson_solve_noalloc runs the same direct solve as
// ibm_poisson_solve with all its workspace (spectrum, residual field,
// twiddle / modified-wavenumber tables, zero-mode buffers, scalars) carved
// from one file-scope __device__ array of kNoAllocBytes.  Every GPU that
// loads this library holds that array until the process exits.
//
// The array is shared by all calls and keeps the previous call's contents;
// every region a solve reads is written earlier in the same call (the error
// word is cleared on entry).  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array; serialise them.
#include <cmath>
#include <mutex>

#include "plan.h"

namespace ibm {

constexpr size_t kNoAllocBytes = (size_t)24 << 20;  // 24 MiB: a 128^3 FP32 solve with refinement

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device (the symbol's
// name in host code is only a stand-in).  Looked up once per device.
static int noalloc_scratch(unsigned char **out) {
  static std::mutex mu;
  static unsigned char *addr[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(IBM_ERR_UNSUPPORTED, "ibm_poisson_solve_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
    addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = addr[dev];
  return IBM_OK;
}

// Twiddles W_N^m and modified wavenumbers (2/h^2)(1 - cos(2 pi k / n))
// (Appendix A), evaluated in FP64 on the device and rounded to FP32; also
// clears the error word.
__global__ void k_noalloc_tables(float2 *twx, int nx, float2 *twz, int nz, float *lamx, int P, float *lamz,
                                 double hx, double hz, int *err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *err = 0;
  if (t < nx) {
    double s, c;
    sincospi(2.0 * t / nx, &s, &c);
    twx[t] = make_float2((float)c, (float)-s);
  }
  if (t < nz) {
    double s, c;
    sincospi(2.0 * t / nz, &s, &c);
    twz[t] = make_float2((float)c, (float)-s);
    lamz[t] = (float)(2.0 / (hz * hz) * (1.0 - cospi(2.0 * t / nz)));
  }
  if (t < P) lamx[t] = (float)(2.0 / (hx * hx) * (1.0 - cospi(2.0 * t / nx)));
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace ibm

using namespace ibm;

extern "C" int ibm_poisson_solve_noalloc(int nx, int ny, int nz, const double h[3], int refine_iters,
                                         const float *rhs, float *phi, int *status, void *stream) {
  if (!h || !rhs || !phi) return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: NULL argument");
  if (!transform_size_supported(nx) || !transform_size_supported(nz))
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: nx=%d nz=%d must be 2^a 3^b (b<=1) in [8,512]",
                     nx, nz);
  if (ny < 8 || ny > 512) return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: ny=%d outside [8,512]", ny);
  if (!(h[0] > 0) || !(h[1] > 0) || !(h[2] > 0) || !std::isfinite(h[0]) || !std::isfinite(h[1]) ||
      !std::isfinite(h[2]))
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: spacings must be finite and positive");
  if (refine_iters < 0 || refine_iters > 4)
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: refine_iters %d outside [0,4]", refine_iters);
  if ((const void *)rhs == (const void *)phi)
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: rhs and phi must be distinct buffers");
  if (!aligned_to(rhs, 16) || !aligned_to(phi, 16))
    return set_error(IBM_ERR_ARG, "ibm_poisson_solve_noalloc: field pointers must be 16-byte aligned");

  const int P = nx / 2 + 1;
  const size_t npts = (size_t)nx * ny * nz;
  const size_t nspec = (size_t)ny * nz * P;
  // carve the scratch: spectrum, residual field, tables, scalars
  size_t off[9], cur = 0;
  const size_t sizes[9] = {nspec * sizeof(float2), refine_iters > 0 ? npts * sizeof(float) : 0,
                           (size_t)nx * sizeof(float2), (size_t)nz * sizeof(float2), (size_t)P * sizeof(float),
                           (size_t)nz * sizeof(float), 16 * sizeof(double), 16, 2 * (size_t)ny * sizeof(double)};
  for (int i = 0; i < 9; ++i) {
    off[i] = cur;
    cur += align256(sizes[i]);
  }
  if (cur > kNoAllocBytes)
    return set_error(IBM_ERR_ARG,
                     "ibm_poisson_solve_noalloc: %dx%dx%d with %d refinement step(s) needs %zu bytes of scratch; "
                     "the static no-alloc scratch holds %zu bytes",
                     nx, ny, nz, refine_iters, cur, kNoAllocBytes);
  unsigned char *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;

  // a plan descriptor on the host stack pointing into the scratch; no device
  // allocation.  Value-initialised: every member plan_solve reaches that is
  // not set below (the periodic-branch tables, the three-field spectra, the
  // tensor-core DFT tables) is null, and the kernels are the ones
  // ibm_plan_create picks for this shape (same boundary kind, plane mode and
  // pencil mode).
  ibm_plan_s p{};
  p.nx = nx; p.ny = ny; p.nz = nz; p.P = P;
  p.bc = IBM_BC_PXZ_WALL_Y;
  p.use_plane = default_plane_mode<float>(nx, ny, nz);
  p.use_slab = default_use_slab(IBM_FP32_REFINED, IBM_BC_PXZ_WALL_Y, nx, ny, nz) ? 1 : 0;
  p.use_plane_fields = 0;
  p.h[0] = h[0]; p.h[1] = h[1]; p.h[2] = h[2];
  p.precision = IBM_FP32_REFINED;
  p.refine = refine_iters;
  p.delta = IBM_DELTA_ROMA3;
  p.pencil_mode = 0;
  p.esz = 4;
  p.npts = npts;
  p.nspec = nspec;
  p.S = base + off[0];
  p.work = refine_iters > 0 ? base + off[1] : nullptr;
  p.bsave = nullptr;
  for (int q = 0; q < 4; ++q) p.sub[q] = nullptr;
  p.mkbuf = nullptr;
  p.mkcap = 0;
  p.twx = base + off[2];
  p.twz = base + off[3];
  p.lamx = base + off[4];
  p.lamz = base + off[5];
  p.dsc = reinterpret_cast<double *>(base + off[6]);
  p.derr = reinterpret_cast<int *>(base + off[7]);
  p.zbuf = reinterpret_cast<double *>(base + off[8]);
  p.hsc = nullptr;
  p.ev0 = p.ev1 = nullptr;
  p.bytes = 0;
  p.prof_on = 0;

  cudaStream_t st = (cudaStream_t)stream;
  const int nt = std::max(std::max(nx, nz), P);
  k_noalloc_tables<<<(nt + 127) / 128, 128, 0, st>>>((float2 *)p.twx, nx, (float2 *)p.twz, nz, (float *)p.lamx, P,
                                                     (float *)p.lamz, h[0], h[2], p.derr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "ibm_poisson_solve_noalloc: table kernel");
  rc = plan_solve(&p, 0, 0.0, 0, rhs, phi, nullptr, st, nullptr);
  if (rc) return rc;
  // the solve's error word (0: every bounded wait completed) to the caller
  if (status) {
    e = cudaMemcpyAsync(status, p.derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "ibm_poisson_solve_noalloc: status copy");
  }
  return IBM_OK;
}
