// stencil.cu -- 7-point residual of the Poisson / Helmholtz operators.
//
// r = b - (sigma x + tau L_h x), L_h the second-order central Laplacian of
// Sec. 2.1 with periodic x, z and the ghost rule of the field's wall kind
// along y (Appendix B; periodic for the triply periodic branch).  Poisson:
// sigma = 0, tau = 1; Helmholtz (I - c L):
// sigma = 1, tau = -c.  In FP32 the second differences of the stored values
// are taken exactly (hi + lo) and the other terms, all O(|b|), are summed in
// FP32 (residual_point below): a plain FP32 stencil would lose the residual
// in the cancelling second differences.  Optionally the
// FP64 sums of r^2, b^2, r and b are accumulated for the relative residual.
// An optional device scalar is subtracted from b first (the Poisson
// right-hand side's removed mean), so the residual is that of the compatible
// system.
#include "stencil.cuh"

namespace ibm {

// Four consecutive x points per thread (residual4).  Grid
// (ceil(nz nx / 4 / 128), ny), 128 threads.
template <int BC, bool SIGMA>
__global__ void __launch_bounds__(128)
k_residual_f32v(ResidualArgs A, const float *__restrict__ b, const float *__restrict__ x, float *__restrict__ r,
                double *norms) {
  pdl_wait();
  const int q = A.nx >> 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  double r2 = 0.0, b2 = 0.0, r1 = 0.0, b1 = 0.0;
  if (t < q * A.nz) {
    const int k = t / q, i0 = 4 * (t - k * q);
    float2 m = make_float2(0.f, 0.f);
    if (A.boff) m = *reinterpret_cast<const float2 *>(A.boff + 1);
    float4 bt;
    const float4 res = residual4<BC, SIGMA>(A, b, x, j, k, i0, m, bt);
    if (norms) residual4_norms(res, bt, r2, b2, r1, b1);
    *reinterpret_cast<float4 *>(r + (size_t)j * A.nx * A.nz + (size_t)k * A.nx + i0) = res;
  }
  if (norms) block_accumulate(r2, b2, r1, b1, norms);
}

__global__ void __launch_bounds__(128)
k_residual_f64(ResidualArgs A, const double *__restrict__ b, const double *__restrict__ x,
               double *__restrict__ r, double *norms) {
  pdl_wait();
  int i, k, j;
  const bool inside = stencil_index(A.nx, A.nz, i, k, j);
  const size_t idx = ((size_t)j * A.nz + k) * A.nx + i;
  double rr = 0.0, bb = 0.0;
  if (inside) {
    const size_t row = (size_t)A.nx;
    const size_t pl = (size_t)A.nx * A.nz;
    const double bv = A.boff ? b[idx] - *A.boff : b[idx];
    double res;
    if (A.bc == BC_FACE_DIRICHLET && j == 0) {
      res = 0.0;
    } else {
      const double x0 = x[idx];
      const double xe = x[idx - i + (i + 1 == A.nx ? 0 : i + 1)];
      const double xw = x[idx - i + (i == 0 ? A.nx - 1 : i - 1)];
      const size_t rowbase = idx - (size_t)k * row;
      const double xn = x[rowbase + (size_t)(k + 1 == A.nz ? 0 : k + 1) * row];
      const double xs = x[rowbase + (size_t)(k == 0 ? A.nz - 1 : k - 1) * row];
      double xu, xd;
      if (A.bc == BC_FACE_DIRICHLET) {
        xd = (j - 1 >= 1) ? x[idx - pl] : 0.0;
        xu = (j + 1 <= A.ny - 1) ? x[idx + pl] : 0.0;
      } else if (A.bc == BC_PERIODIC) {
        xd = j > 0 ? x[idx - pl] : x[idx + (size_t)(A.ny - 1) * pl];
        xu = j + 1 < A.ny ? x[idx + pl] : x[idx - (size_t)(A.ny - 1) * pl];
      } else {
        const double gsign = (A.bc == BC_NEUMANN) ? 1.0 : -1.0;
        xd = (j > 0) ? x[idx - pl] : gsign * x0;
        xu = (j + 1 < A.ny) ? x[idx + pl] : gsign * x0;
      }
      const double L = (xe + xw - 2.0 * x0) * A.cxd + (xn + xs - 2.0 * x0) * A.czd + (xu + xd - 2.0 * x0) * A.cyd;
      res = bv - A.sigmad * x0 - A.taud * L;
    }
    r[idx] = res;
    rr = res;
    bb = (A.bc == BC_FACE_DIRICHLET && j == 0) ? 0.0 : bv;
  }
  if (norms) block_accumulate(rr * rr, bb * bb, rr, bb, norms);
}


template <int BC, bool SIGMA>
static cudaError_t launch_residual_f32(const ResidualArgs &A, const float *b, const float *x, float *r, double *norms,
                                       cudaStream_t st) {
  const int units = A.nz * (A.nx / 4);
  IBM_KTRY(launch_pdl(k_residual_f32v<BC, SIGMA>, dim3((unsigned)ceil_div(units, 128), (unsigned)A.ny), 128, 0, st, A,
                      b, x, r, norms));
  return cudaGetLastError();
}

template <>
cudaError_t launch_residual<float>(int nx, int ny, int nz, const StencilCoef &c, const float *b, const float *x,
                                   float *r, const double *boff, double *norms, cudaStream_t st) {
  if (nx % 4 != 0 || ((uintptr_t)b | (uintptr_t)x | (uintptr_t)r) & 15u) return cudaErrorInvalidValue;
  const ResidualArgs A = make_args(nx, ny, nz, c, boff);
  const bool sg = c.sigma != 0.0;
#define IBM_RES_BC(B)                                                                             \
  case B:                                                                                         \
    return sg ? launch_residual_f32<B, true>(A, b, x, r, norms, st) : launch_residual_f32<B, false>(A, b, x, r, norms, st);
  switch (c.bc) {
    IBM_RES_BC(BC_NEUMANN)
    IBM_RES_BC(BC_CELL_DIRICHLET)
    IBM_RES_BC(BC_FACE_DIRICHLET)
    IBM_RES_BC(BC_PERIODIC)
    default: return cudaErrorInvalidValue;
  }
#undef IBM_RES_BC
}

// Wall data's share of the 7-point operator, moved to the right-hand side
// (Appendix B: the first and last rows of each pencil carry the boundary
// values; BC2.2 forms the same terms from the FFT of the ghost planes).
// dst[jlo] += clo g_lo, dst[jhi] += chi g_hi over one x-z plane each (either
// g may be NULL).  One thread per plane point.
template <typename T>
__global__ void __launch_bounds__(256)
k_wall_rhs(int npl, T *dst, size_t plane, int jlo, int jhi, const T *glo, const T *ghi, T clo, T chi) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npl) return;
  if (glo) dst[(size_t)jlo * plane + i] += clo * glo[i];
  if (ghi) dst[(size_t)jhi * plane + i] += chi * ghi[i];
}

template <typename T>
cudaError_t launch_wall_rhs(int nx, int nz, T *dst, int jlo, int jhi, const T *glo, const T *ghi, double clo,
                            double chi, cudaStream_t st) {
  const int npl = nx * nz;
  IBM_KTRY(launch_pdl(k_wall_rhs<T>, ceil_div(npl, 256), 256, 0, st, npl, dst, (size_t)npl, jlo, jhi, glo, ghi,
                      (T)clo, (T)chi));
  return cudaGetLastError();
}
template cudaError_t launch_wall_rhs<float>(int, int, float *, int, int, const float *, const float *, double, double,
                                            cudaStream_t);
template cudaError_t launch_wall_rhs<double>(int, int, double *, int, int, const double *, const double *, double,
                                             double, cudaStream_t);

template <>
cudaError_t launch_residual<double>(int nx, int ny, int nz, const StencilCoef &c, const double *b, const double *x,
                                    double *r, const double *boff, double *norms, cudaStream_t st) {
  const Launch3 L = stencil_launch(nx, ny, nz);
  IBM_KTRY(launch_pdl(k_residual_f64, L.grid, L.block, 0, st, make_args(nx, ny, nz, c, boff), b, x, r, norms));
  return cudaGetLastError();
}

}  // namespace ibm
