// internal.h -- declarations shared by the libibm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace ibm {

// Largest dynamic shared memory a plane kernel may take (bytes).
constexpr size_t kPlaneSmemLimit = 227 * 1024;

// Up to three fields of one grid moved through the same launches (the
// three velocity components of a Helmholtz stage); a kernel picks its field
// by blockIdx.y.
constexpr int kMaxFields = 3;
template <typename P> struct Ptr3 {
  P p[kMaxFields];
  __host__ __device__ __forceinline__ P operator[](int b) const { return b == 0 ? p[0] : (b == 1 ? p[1] : p[2]); }
};
template <typename P> inline Ptr3<P> ptr3(P a, P b = nullptr, P c = nullptr) { return Ptr3<P>{{a, b, c}}; }

struct TransformGeom {
  int nx, ny, nz;
  int nb;          // fields in the launch (1..kMaxFields)
  int use_plane;   // plane mode: 0 split x / z passes; 1 one CTA per plane; C >= 2 a cluster of C CTAs per plane;
                   // kPlaneDft tensor-core DFT products
  int *err;        // device error word for bounded waits
  double *zrhs;    // forward: if set, receives Re S[j][0][0] of every plane (the zero pencil)
  const double *zsol;  // inverse: if set, replaces S[j][0][0] by (zsol[j], 0) before transforming
  const void *dft_fwd, *dft_inv;  // plane mode kPlaneDft: the DFT matrix tables (FP32 plans)
};

// Plane mode of the tensor-core DFT transforms (dft_tc.cu).
constexpr int kPlaneDft = -1;

// Lanes that exist in the calling thread's warp (a block of fewer than 32
// threads has a partial last warp).
__device__ __forceinline__ unsigned warp_full_mask() {
  const int warp_base = (threadIdx.x / 32) * 32;
  const int lanes = min(32, (int)blockDim.x - warp_base);
  return lanes >= 32 ? 0xffffffffu : ((1u << lanes) - 1u);
}

// Launch shape of the point-wise stencil kernels: threads along x (coalesced),
// grid over (x blocks, z, y); no index divisions in the kernels.
struct Launch3 {
  dim3 grid, block;
};
inline Launch3 stencil_launch(int nx, int ny, int nz) {
  const int bx = nx >= 128 ? 128 : 32;
  const int bz = 128 / bx;
  return {dim3((unsigned)ceil_div(nx, bx), (unsigned)ceil_div(nz, bz), (unsigned)ny), dim3(bx, bz, 1)};
}
// (i, k, j) of the calling thread under stencil_launch; false if outside.
__device__ __forceinline__ bool stencil_index(int nx, int nz, int &i, int &k, int &j) {
  i = blockIdx.x * blockDim.x + threadIdx.x;
  k = blockIdx.y * blockDim.y + threadIdx.y;
  j = blockIdx.z;
  return i < nx && k < nz;
}

// Raises a kernel's dynamic shared-memory limit to the per-block maximum,
// once per kernel and thread-safely (plans on several host threads may make
// the first launch concurrently).  The limit does not change occupancy; the
// launch's actual request does.
template <auto Kernel> cudaError_t ensure_max_smem() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlaneSmemLimit);
  });
  return err;
}

// Programmatic dependent launch.  Every kernel of the path is launched
// with programmatic stream serialization: the next kernel in the stream may
// be launched once every CTA of this one has exited (the implicit trigger),
// which overlaps its launch and prologue with this grid's completion.
// Before it touches memory written by its predecessor each kernel waits for
// that grid's completion (griddepcontrol.wait, which also orders memory);
// only plan constants (twiddle and wavenumber tables) are read before the
// wait.  No kernel triggers early: dependents scheduled while a many-wave
// grid still has CTAs to run would take its SM slots (measured: the E2
// divergence at 256^3 ran at half speed).  IBM_PDL=0 turns the attribute
// off (plain stream order; the wait is then a no-op).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Returns a failed launch's error from a function returning cudaError_t.
#define IBM_KTRY(call)                          \
  do {                                          \
    cudaError_t e__ = (call);                   \
    if (e__ != cudaSuccess) return e__;         \
  } while (0)

bool transform_size_supported(int n);
// Plane modes (kPlaneDft, 0, 1, 2, 4, 8) that can run an nx x nz plane; returns the count.
template <typename T> int plane_modes(int nx, int nz, int *modes);
// Plane mode used when no tuning result is known.
template <typename T> int default_plane_mode(int nx, int ny, int nz);
// Kernels one forward (or inverse) transform launches: 1 on the plane path, 2 otherwise.
template <typename T> int transform_launches(const TransformGeom &g);

// Forward: real field [ny][nz][nx] (times in_scale) -> spectrum [ny][nz][nx/2+1],
// for fields 0 .. g.nb-1.
template <typename T>
cudaError_t launch_forward(const TransformGeom &g, Ptr3<const T *> in, Ptr3<cplx<T> *> S, const cplx<T> *twx,
                           const cplx<T> *twz, T in_scale, cudaStream_t st);
// Inverse: spectrum -> out = addend + scale * field (addend may be NULL or equal out).
template <typename T>
cudaError_t launch_inverse(const TransformGeom &g, Ptr3<cplx<T> *> S, Ptr3<T *> out, Ptr3<const T *> addend,
                           const cplx<T> *twx, const cplx<T> *twz, T scale, cudaStream_t st);

// Tensor-core DFT plane transforms (FP32; nx, nz in {8, 16, 24, 32, 48, 64}):
// the same contracts as launch_forward / launch_inverse.
bool dft_tc_supported(int nx, int nz);
cudaError_t dft_tc_upload(int nx, int nz, void **fwd, void **inv, size_t *bytes);
cudaError_t launch_dft_forward(const TransformGeom &g, Ptr3<const float *> in, Ptr3<float2 *> S, float in_scale,
                               cudaStream_t st);
cudaError_t launch_dft_inverse(const TransformGeom &g, Ptr3<float2 *> S, Ptr3<float *> out,
                               Ptr3<const float *> addend, float scale, cudaStream_t st);

// Split passes: x rows then z columns (forward), z columns then x rows (inverse).
template <typename T>
cudaError_t launch_axis_forward(const TransformGeom &g, Ptr3<const T *> in, Ptr3<cplx<T> *> S, const cplx<T> *twx,
                                const cplx<T> *twz, T in_scale, cudaStream_t st);
template <typename T>
cudaError_t launch_axis_inverse(const TransformGeom &g, Ptr3<cplx<T> *> S, Ptr3<T *> out, Ptr3<const T *> addend,
                                const cplx<T> *twx, const cplx<T> *twz, T scale, cudaStream_t st);

// Cluster plane kernels (C CTAs per y-plane, rows and columns exchanged
// through distributed shared memory); cudaErrorNotSupported for shapes
// without an instantiation.
template <typename T> bool cplane_supported(int nx, int nz, int C);
template <typename T>
cudaError_t launch_cplane_forward(const TransformGeom &g, int C, Ptr3<const T *> in, Ptr3<cplx<T> *> S,
                                  const cplx<T> *twx, const cplx<T> *twz, T in_scale, cudaStream_t st);
template <typename T>
cudaError_t launch_cplane_inverse(const TransformGeom &g, int C, Ptr3<cplx<T> *> S, Ptr3<T *> out,
                                  Ptr3<const T *> addend, const cplx<T> *twx, const cplx<T> *twz, T scale,
                                  cudaStream_t st);

// Pencil solve along y (Thomas, excess form), in place on the spectrum.
struct PencilParams {
  int ny, nz, P;           // P = nx/2 + 1
  double a;                // off-diagonal magnitude of M = tridiag(-a, ., -a)
  double g_add, g_mul;     // g = g_add + g_mul (lambda_x + lambda_z)
  int beta_s, beta_e;      // wall rows: first diag = a(1+beta_s) + g
  int j0;                  // first unknown plane (1 for wall-normal faces)
  int neg_rhs;             // solve M x = -rhs (Poisson: M = -L)
  int zero_mode;           // Poisson: solve the (0,0) pencil in FP64
  double hy2;              // hy^2 for the FP64 zero-mode path
  double inv_nxnz;         // 1/(nx nz) for the removed-mean report
  int *err;                // device error word for bounded waits
  int mode;                // pencil kernel: 0 auto (FP32: segmented where ny allows; else tile or
                           // streaming by size), 1 warp-parallel block solve (n <= 256 FP32 / 128
                           // FP64, else auto), 2 tile, 3 streaming, 4 segmented (ny <= 512 FP32 / 256
                           // FP64)
  const double *zrhs;      // zero_mode: right-hand side of the (0,0) pencil, [ny] (from the forward pass)
  double *zsol;            // zero_mode: its FP64 solution, [ny] (read by the inverse pass)
  double inv_ny;           // 1/ny
  int periodic;            // triply periodic branch: y-transform + divide (twy, lamy) instead of Thomas
  const void *twy;         // periodic: W_ny^m twiddles (plan precision)
  const void *lamy;        // periodic: lambda_y(ky) (plan precision)
  int nb;                  // fields in the launch; field b > 0 takes its wall rows from fbc[b]
  int fbc[kMaxFields];     // beta_s | beta_e << 4 | j0 << 8 of each field
};
// Wall-row parameters of field b (blockIdx.y) of a pencil launch.
__device__ __forceinline__ void pencil_field(const PencilParams &pp, int b, int &beta_s, int &beta_e, int &j0) {
  beta_s = pp.beta_s; beta_e = pp.beta_e; j0 = pp.j0;
  if (b > 0) {
    const int c = b == 1 ? pp.fbc[1] : pp.fbc[2];
    beta_s = c & 15; beta_e = (c >> 4) & 15; j0 = c >> 8;
  }
}
template <typename T>
cudaError_t launch_pencil(const PencilParams &pp, Ptr3<cplx<T> *> S, const T *lamx, const T *lamz, double *mean_out,
                          cudaStream_t st);
// The triply periodic branch's pencil step (periodic.cu).
template <typename T>
cudaError_t launch_ypencil(const PencilParams &pp, Ptr3<cplx<T> *> S3, const cplx<T> *twy, const T *lamx,
                           const T *lamz, const T *lamy, double *mean_out, cudaStream_t st);

// The fused FP32 solve (slab.cu) for wall-bounded grids with ny and nz in
// {64, 128, 256}: phase 0 the x rows forward into the kx-major spectrum
// S[kx][y][z], phase 1 the slab kernel (z transforms and the y sweep of one
// kx slab per cluster, the FP64 zero mode included), phase 2 the x rows
// inverse (out = scale x, or out += scale x when addend == out; any other
// addend is cudaErrorInvalidValue).  Single fields with unknowns on every
// row (j0 = 0) only.
bool slab_supported(int nx, int ny, int nz);
cudaError_t launch_slab_solve(const PencilParams &pp, int nx, const float *in, float2 *S, float *out,
                              const float *addend, const float2 *twx, const float2 *twz, const float *lamx,
                              const float *lamz, double *mean_out, float scale, cudaStream_t st, int phase);

// Residual r = b - (sigma x + tau L x) with float-float arithmetic for FP32.
struct StencilCoef {
  double cx, cy, cz;  // 1/h^2 per axis
  double sigma, tau;
  int bc;             // field boundary kind along y
};
template <typename T>
cudaError_t launch_residual(int nx, int ny, int nz, const StencilCoef &c, const T *b, const T *x, T *r,
                            const double *boff, double *norms, cudaStream_t st);
// The slab path's refinement pass (slab.cu): the FP32 residual r = b - A x
// of the coefficients c (wall kinds IBM_FIELD_CELL_NEUMANN and
// IBM_FIELD_CELL_DIRICHLET) and its forward x rows into the kx-major spectrum
// S, as launch_residual followed by launch_slab_solve phase 0 but without
// storing r.  boff / norms as for launch_residual; err: the plan's device
// error word (bounded waits of the streaming form, 256-point x rows).
bool slab_residual_fused(int nx, int nz);  // the pass exists for this x length (every CTA's rows in one y plane)
cudaError_t launch_slab_residual_forward(const StencilCoef &c, int nx, int ny, int nz, const float *b, const float *x,
                                         float2 *S, const float2 *twx, const double *boff, double *norms, int *err,
                                         cudaStream_t st);
// dst plane jlo += clo g_lo, plane jhi += chi g_hi ([nz][nx] planes; NULL skips a side).
template <typename T>
cudaError_t launch_wall_rhs(int nx, int nz, T *dst, int jlo, int jhi, const T *glo, const T *ghi, double clo,
                            double chi, cudaStream_t st);

}  // namespace ibm
