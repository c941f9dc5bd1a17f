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
#include "internal.h"

namespace ibm {

enum { BC_NEUMANN = 0, BC_CELL_DIRICHLET = 1, BC_FACE_DIRICHLET = 2, BC_PERIODIC = 3 };

struct ffc { float hi, lo; };
static inline ffc split_ff(double v) {
  ffc r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

struct ResidualArgs {
  const double *boff;  // device scalars: boff[0] mean to subtract from b (FP64 path); boff[1] holds the
                       // same value as a float pair (hi, lo) for the FP32 path; NULL for none
  int nx, ny, nz, bc;
  ffc cx, cy, cz, tau;
  ffc kx, ky, kz;  // -tau c_a, split from the FP64 product
  float sigma;
  double cxd, cyd, czd, taud, sigmad;
};

// Adds the block sums of the per-thread sums (r^2, b^2, r, b) to out[0..3]
// (FP64 atomics).
__device__ __forceinline__ void block_accumulate(double r2, double b2, double r1, double b1, double *out) {
  __shared__ double red[4][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  double v[4] = {r2, b2, r1, b1};
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][w] = v[q];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double t = lane < nw ? red[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) atomicAdd(out + q, t);
    }
  }
}

// FP32 residual.  The value
//   r = (b - m) - sigma x0 + sum_a K_a D_a,   K_a = -tau c_a,
// D_a = x(+1) + x(-1) - 2 x0 the second difference along axis a.  The
// second differences are where a plain FP32 stencil loses the residual:
// the stored values are O(|x|) and cancel to O(h^2 |x''|).  They are taken
// exactly, as hi + lo (two error-free sums of FP32 values).  Every other
// term is O(|b|) and is summed in FP32 (K_a as its FP64 value split into
// hi + lo, the small products first): a few FP32 roundings of |b|, against
// a residual of an FP32 solution that is 1e-5 .. 1e-3 of |b| (its rounding
// errors are grid-scale, which L_h amplifies by ~1/h^2), so the correction
// is accurate to better than 1 % and the refined solution reaches the FP32
// rounding of its storage.
template <bool SIGMA>
__device__ __forceinline__ float residual_point(const ResidualArgs &A, float bv, float2 m, float x0, float xe, float xw,
                                                float xn, float xs, float xu, float xd, float &bt) {
  const float x2 = -2.0f * x0;
  // exact second differences D = hi + lo
  ff s = two_sum(xe, xw), t = two_sum(s.hi, x2);
  const float Dxh = t.hi, Dxl = t.lo + s.lo;
  s = two_sum(xn, xs); t = two_sum(s.hi, x2);
  const float Dzh = t.hi, Dzl = t.lo + s.lo;
  s = two_sum(xu, xd); t = two_sum(s.hi, x2);
  const float Dyh = t.hi, Dyl = t.lo + s.lo;
  const float bm = (bv - m.x) - m.y;
  bt = bm;
  float E = fmaf(A.kx.hi, Dxl, A.kx.lo * Dxh);
  E = fmaf(A.kz.hi, Dzl, fmaf(A.kz.lo, Dzh, E));
  E = fmaf(A.ky.hi, Dyl, fmaf(A.ky.lo, Dyh, E));
  float S = SIGMA ? fmaf(-A.sigma, x0, bm) : bm;
  S = fmaf(A.kx.hi, Dxh, S);
  S = fmaf(A.kz.hi, Dzh, S);
  S = fmaf(A.ky.hi, Dyh, S);
  return S + E;
}

// Four consecutive x points per thread (every supported nx is a multiple of
// 4 and the ABI takes 16-byte aligned fields): every row access is a float4,
// the x neighbours of the four come from the same float4 plus two scalars,
// and the index arithmetic is shared.  Grid (ceil(nz nx / 4 / 128), ny), 128
// threads.
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
    const size_t pl = (size_t)A.nx * A.nz;
    const size_t at = (size_t)j * pl + (size_t)k * A.nx + i0;
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!(BC == BC_FACE_DIRICHLET && j == 0)) {
      const size_t row = at - i0;
      const float4 x0 = *reinterpret_cast<const float4 *>(x + at);
      const float xW = x[row + (i0 == 0 ? A.nx - 1 : i0 - 1)];
      const float xE = x[row + (i0 + 4 == A.nx ? 0 : i0 + 4)];
      const long dn = (long)(k + 1 == A.nz ? -(long)(A.nz - 1) * A.nx : (long)A.nx);
      const long ds = (long)(k == 0 ? (long)(A.nz - 1) * A.nx : -(long)A.nx);
      const float4 xn = *reinterpret_cast<const float4 *>(x + at + dn);
      const float4 xs = *reinterpret_cast<const float4 *>(x + at + ds);
      float4 xd, xu;
      if (BC == BC_FACE_DIRICHLET) {
        xd = j - 1 >= 1 ? *reinterpret_cast<const float4 *>(x + at - pl) : make_float4(0.f, 0.f, 0.f, 0.f);
        xu = j + 1 <= A.ny - 1 ? *reinterpret_cast<const float4 *>(x + at + pl) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else if (BC == BC_PERIODIC) {
        xd = *reinterpret_cast<const float4 *>(x + (j > 0 ? at - pl : at + (size_t)(A.ny - 1) * pl));
        xu = *reinterpret_cast<const float4 *>(x + (j + 1 < A.ny ? at + pl : at - (size_t)(A.ny - 1) * pl));
      } else {
        const float gs = BC == BC_NEUMANN ? 1.0f : -1.0f;
        xd = j > 0 ? *reinterpret_cast<const float4 *>(x + at - pl)
                   : make_float4(gs * x0.x, gs * x0.y, gs * x0.z, gs * x0.w);
        xu = j + 1 < A.ny ? *reinterpret_cast<const float4 *>(x + at + pl)
                          : make_float4(gs * x0.x, gs * x0.y, gs * x0.z, gs * x0.w);
      }
      const float4 bv = *reinterpret_cast<const float4 *>(b + at);
      float2 m = make_float2(0.f, 0.f);
      if (A.boff) m = *reinterpret_cast<const float2 *>(A.boff + 1);
      float bt0, bt1, bt2, bt3;
      res.x = residual_point<SIGMA>(A, bv.x, m, x0.x, x0.y, xW, xn.x, xs.x, xu.x, xd.x, bt0);
      res.y = residual_point<SIGMA>(A, bv.y, m, x0.y, x0.z, x0.x, xn.y, xs.y, xu.y, xd.y, bt1);
      res.z = residual_point<SIGMA>(A, bv.z, m, x0.z, x0.w, x0.y, xn.z, xs.z, xu.z, xd.z, bt2);
      res.w = residual_point<SIGMA>(A, bv.w, m, x0.w, xE, x0.z, xn.w, xs.w, xu.w, xd.w, bt3);
      if (norms) {
        r2 = (double)res.x * res.x + (double)res.y * res.y + (double)res.z * res.z + (double)res.w * res.w;
        b2 = (double)bt0 * bt0 + (double)bt1 * bt1 + (double)bt2 * bt2 + (double)bt3 * bt3;
        r1 = (double)res.x + res.y + res.z + res.w;
        b1 = (double)bt0 + bt1 + bt2 + bt3;
      }
    }
    *reinterpret_cast<float4 *>(r + at) = res;
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

static ResidualArgs make_args(int nx, int ny, int nz, const StencilCoef &c, const double *boff) {
  ResidualArgs A;
  A.boff = boff;
  A.nx = nx; A.ny = ny; A.nz = nz; A.bc = c.bc;
  A.cx = split_ff(c.cx); A.cy = split_ff(c.cy); A.cz = split_ff(c.cz);
  A.tau = split_ff(c.tau);
  A.kx = split_ff(-c.tau * c.cx); A.ky = split_ff(-c.tau * c.cy); A.kz = split_ff(-c.tau * c.cz);
  A.sigma = (float)c.sigma;
  A.cxd = c.cx; A.cyd = c.cy; A.czd = c.cz; A.taud = c.tau; A.sigmad = c.sigma;
  return A;
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
