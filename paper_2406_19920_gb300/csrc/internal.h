// internal.h -- declarations shared by the libibm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace ibm {

// Largest dynamic shared memory a plane kernel may take (bytes).
constexpr size_t kPlaneSmemLimit = 200 * 1024;

struct TransformGeom {
  int nx, ny, nz;
  bool use_plane;  // allow the one-CTA-per-plane kernels
};

// Lanes that exist in the calling thread's warp (a block of fewer than 32
// threads has a partial last warp).
__device__ __forceinline__ unsigned warp_full_mask() {
  const int warp_base = (threadIdx.x / 32) * 32;
  const int lanes = min(32, (int)blockDim.x - warp_base);
  return lanes >= 32 ? 0xffffffffu : ((1u << lanes) - 1u);
}

bool transform_size_supported(int n);
// Kernels one forward (or inverse) transform launches: 1 on the plane path, 2 otherwise.
template <typename T> int transform_launches(const TransformGeom &g);

// Forward: real field [ny][nz][nx] (times in_scale) -> spectrum [ny][nz][nx/2+1].
template <typename T>
cudaError_t launch_forward(const TransformGeom &g, const T *in, cplx<T> *S, const cplx<T> *twx,
                           const cplx<T> *twz, T in_scale, cudaStream_t st);
// Inverse: spectrum -> out = addend + scale * field (addend may be NULL or equal out).
template <typename T>
cudaError_t launch_inverse(const TransformGeom &g, cplx<T> *S, T *out, const T *addend, const cplx<T> *twx,
                           const cplx<T> *twz, T scale, cudaStream_t st);

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
};
template <typename T>
cudaError_t launch_pencil(const PencilParams &pp, cplx<T> *S, const T *lamx, const T *lamz, double *mean_out,
                          cudaStream_t st);

// Residual r = b - (sigma x + tau L x) with float-float arithmetic for FP32.
struct StencilCoef {
  double cx, cy, cz;  // 1/h^2 per axis
  double sigma, tau;
  int bc;             // field boundary kind along y
};
template <typename T>
cudaError_t launch_residual(int nx, int ny, int nz, const StencilCoef &c, const T *b, const T *x, T *r,
                            const double *boff, double *norms, cudaStream_t st);

}  // namespace ibm
