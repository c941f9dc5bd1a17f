// ibm_kernels.cu -- Lagrangian operations of the immersed boundary (Sec. 2.3.2).
//
// Interpolation (Eq. 2b) and spreading (Eq. 2d) with a regularised delta
// delta_h(x - X) = phi((x-X)/hx) phi((y-Y)/hy) phi((z-Z)/hz) / (hx hy hz).
// The paper cites Peskin and Roma et al. without printing phi; ROMA3 is the
// three-point kernel of Roma, Peskin & Berger (1999), PESKIN4 the four-point
// kernel of Peskin (2002).  Each velocity component lives on its own
// staggered sub-grid (origin in grid units: u (0,1/2,1/2), v (1/2,0,1/2),
// w (1/2,1/2,0)); x and z wrap periodically; along y only stored unknowns
// are touched (v's wall face 0 and points beyond the walls are dropped).
//
// One thread per (marker, component).  The stencil origin and offset are
// computed in FP64 on the FP64 path and in float-float on the FP32 path, so
// that the weights see the marker position without the FP32 rounding of
// X/h; the weights and sums run in the plan precision.  Spreading
// accumulates with global atomics as in the paper's L1 kernel (Sec. 2.3.2).
#include <cmath>

#include "plan.h"

namespace ibm {

struct IbmGrid {
  int nx, ny, nz;
  double inv_h[3];
  float ih_hi[3], ih_lo[3];  // 1/h as float-float for the FP32 path
  double vol_inv;            // 1 / (hx hy hz)
};

// L2 for the rigid motions (Sec. 2.3.2 moves the markers before L1): every
// marker is displaced by the same d(t) with velocity v(t), both evaluated on
// the host in FP64; d also as a float-float pair for the FP32 path.
struct RigidMotion {
  double d[3], v[3];
  float dh[3], dl[3];
};

// X0 + d rounded once to the working precision.
__device__ __forceinline__ double displaced(double x0, const RigidMotion &mo, int c) { return x0 + mo.d[c]; }
__device__ __forceinline__ float displaced(float x0, const RigidMotion &mo, int c) {
  const ff s = two_sum(x0, mo.dh[c]);
  return s.hi + (s.lo + mo.dl[c]);
}

template <typename T> __device__ __forceinline__ T phi_roma3(T r) {
  const T a = fabs(r);
  if (a <= (T)0.5) return ((T)1 + sqrt((T)1 - (T)3 * a * a)) / (T)3;
  if (a <= (T)1.5) {
    const T t = (T)1 - a;
    return ((T)5 - (T)3 * a - sqrt(fmax((T)0, (T)1 - (T)3 * t * t))) / (T)6;
  }
  return (T)0;
}
template <typename T> __device__ __forceinline__ T phi_peskin4(T r) {
  const T a = fabs(r);
  if (a <= (T)1) return ((T)3 - (T)2 * a + sqrt((T)1 + (T)4 * a - (T)4 * a * a)) / (T)8;
  if (a <= (T)2) return ((T)5 - (T)2 * a - sqrt(fmax((T)0, (T)-7 + (T)12 * a - (T)4 * a * a))) / (T)8;
  return (T)0;
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Stencil origin along one axis: s = X/h - o in grid units, first index b
// and offset f = s - b.  FP64: plain doubles.  FP32: s as a float-float (an
// error-free product of X with 1/h split into hi + lo, and an error-free
// sum for the half-cell shift), b from its high part, f = (hi - b) + lo;
// f is within about 1e-7 grid units of the exact offset, and no FP64
// instruction is issued (the FP64 pipe is narrow on this part).
template <int S> __device__ __forceinline__ void axis_origin(double X, double ih, float, float, double o, int &b, double &f) {
  const double sx = X * ih - o;
  const double d = (S == 3) ? floor(sx + 0.5) - 1.0 : floor(sx) - 1.0;
  b = (int)d;
  f = sx - d;
}
template <int S> __device__ __forceinline__ void axis_origin(float X, double, float ihh, float ihl, double o, int &b, float &f) {
  const ff p = two_prod(X, ihh);
  const ff t = two_sum(p.hi, -(float)o);
  const float lo = fmaf(X, ihl, p.lo) + t.lo;
  const float hi = t.hi;
  const float d = (S == 3) ? floorf(hi + 0.5f) - 1.0f : floorf(hi) - 1.0f;
  b = (int)d;
  f = (hi - d) + lo;
}

// Component comp's stencil origin (b*) and offsets from it (f*, grid units).
template <typename T, int S>
__device__ __forceinline__ void stencil_origin(const IbmGrid &g, int comp, T X, T Y, T Z, int &bx, int &by, int &bz,
                                               T &fx, T &fy, T &fz) {
  axis_origin<S>(X, g.inv_h[0], g.ih_hi[0], g.ih_lo[0], comp == 0 ? 0.0 : 0.5, bx, fx);
  axis_origin<S>(Y, g.inv_h[1], g.ih_hi[1], g.ih_lo[1], comp == 1 ? 0.0 : 0.5, by, fy);
  axis_origin<S>(Z, g.inv_h[2], g.ih_hi[2], g.ih_lo[2], comp == 2 ? 0.0 : 0.5, bz, fz);
}

// One thread per (marker, component): the whole S^3 stencil of one
// component (its S^3 accesses independent of each other, so they overlap).
// With X0 (the substep): the marker's position X = X0 + d and surface
// velocity Ud = v are formed here (L2), written out, and used at once; the
// CTA's 64 markers share their coordinates through shared memory.  Without
// X0 (ibm_interp): X is read.
constexpr int kMarkerThreads = 192;  // a multiple of 3 and of the warp

template <typename T, int S>
__global__ void __launch_bounds__(kMarkerThreads)
k_interp(IbmGrid g, int n, const T *X, const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ w,
         const T *__restrict__ du, const T *__restrict__ dv, const T *__restrict__ dw, T *__restrict__ U,
         const T *Ud, T inv_dt, T *__restrict__ F, const T *__restrict__ X0, T *Xout, T *Udout, RigidMotion mo) {
  __shared__ T xs[kMarkerThreads];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = t / 3, c = t - 3 * m;
  T ud_c = (T)0;
  if (X0) {
    T xc = (T)0;
    if (t < 3 * n) {
      xc = (T)displaced(X0[t], mo, c);  // X0 is a caller constant: read before the wait
      ud_c = (T)mo.v[c];
    }
    xs[threadIdx.x] = xc;
    __syncthreads();
  }
  pdl_wait();
  if (t >= 3 * n) return;
  if (X0) {
    Xout[t] = xs[threadIdx.x];
    Udout[t] = ud_c;
  }
  const int ml = threadIdx.x - c;  // this marker's first thread in the CTA
  const T mx = X0 ? xs[ml] : X[3 * m], my = X0 ? xs[ml + 1] : X[3 * m + 1], mz = X0 ? xs[ml + 2] : X[3 * m + 2];
  int bx, by, bz;
  T fx, fy, fz;
  stencil_origin<T, S>(g, c, mx, my, mz, bx, by, bz, fx, fy, fz);
  const T *f = c == 0 ? u : c == 1 ? v : w;
  const T *df = c == 0 ? du : c == 1 ? dv : dw;
  T wx[S], wz[S];
  int ix[S], kz[S];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    wx[q] = S == 3 ? phi_roma3<T>(fx - (T)q) : phi_peskin4<T>(fx - (T)q);
    wz[q] = S == 3 ? phi_roma3<T>(fz - (T)q) : phi_peskin4<T>(fz - (T)q);
    ix[q] = wrap(bx + q, g.nx);
    kz[q] = wrap(bz + q, g.nz);
  }
  const int jlo = c == 1 ? 1 : 0;
  T acc = 0;
#pragma unroll
  for (int qy = 0; qy < S; ++qy) {
    const int j = by + qy;
    if (j < jlo || j > g.ny - 1) continue;
    const T wy = S == 3 ? phi_roma3<T>(fy - (T)qy) : phi_peskin4<T>(fy - (T)qy);
#pragma unroll
    for (int qz = 0; qz < S; ++qz) {
      const int row = (j * g.nz + kz[qz]) * g.nx;
      T part = 0;
#pragma unroll
      for (int qx = 0; qx < S; ++qx) {
        T val = f[row + ix[qx]];
        if (df) val += df[row + ix[qx]];
        part += wx[qx] * val;
      }
      acc += wy * wz[qz] * part;
    }
  }
  if (U) U[t] = acc;
  if (F) F[t] = ((X0 ? ud_c : Ud[t]) - acc) * inv_dt;  // Eq. 2c
}

template <typename T, int S>
__global__ void __launch_bounds__(256)
k_spread(IbmGrid g, int n, const T *__restrict__ X, const T *__restrict__ F, const T *__restrict__ dV, T *fu,
           T *fv, T *fw, T scale) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int m = t / 3, c = t - 3 * m;
  int bx, by, bz;
  T fx, fy, fz;
  stencil_origin<T, S>(g, c, X[3 * m], X[3 * m + 1], X[3 * m + 2], bx, by, bz, fx, fy, fz);
  T *f = c == 0 ? fu : c == 1 ? fv : fw;
  const T amp = scale * F[t] * dV[m] * (T)g.vol_inv;
  T wx[S], wz[S];
  int ix[S], kz[S];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    wx[q] = S == 3 ? phi_roma3<T>(fx - (T)q) : phi_peskin4<T>(fx - (T)q);
    wz[q] = S == 3 ? phi_roma3<T>(fz - (T)q) : phi_peskin4<T>(fz - (T)q);
    ix[q] = wrap(bx + q, g.nx);
    kz[q] = wrap(bz + q, g.nz);
  }
  const int jlo = c == 1 ? 1 : 0;
#pragma unroll
  for (int qy = 0; qy < S; ++qy) {
    const int j = by + qy;
    if (j < jlo || j > g.ny - 1) continue;
    const T wy = S == 3 ? phi_roma3<T>(fy - (T)qy) : phi_peskin4<T>(fy - (T)qy);
#pragma unroll
    for (int qz = 0; qz < S; ++qz) {
      const int row = (j * g.nz + kz[qz]) * g.nx;
      const T a = amp * wy * wz[qz];
#pragma unroll
      for (int qx = 0; qx < S; ++qx) atomicAdd(f + row + ix[qx], a * wx[qx]);
    }
  }
}

static IbmGrid ibm_grid(const ibm_plan_s *p) {
  IbmGrid g;
  g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
  for (int d = 0; d < 3; ++d) {
    g.inv_h[d] = 1.0 / p->h[d];
    g.ih_hi[d] = (float)g.inv_h[d];
    g.ih_lo[d] = (float)(g.inv_h[d] - (double)g.ih_hi[d]);
  }
  g.vol_inv = 1.0 / (p->h[0] * p->h[1] * p->h[2]);
  return g;
}

// Rigid-motion displacement and velocity at time t (FP64, host).
static RigidMotion rigid_motion(int kind, const double *params, double t) {
  RigidMotion mo = {};
  if (kind == IBM_MOTION_TRANSLATE) {
    for (int c = 0; c < 3; ++c) { mo.d[c] = params[c] * t; mo.v[c] = params[c]; }
  } else if (kind == IBM_MOTION_HEAVE) {
    const double w = 2.0 * M_PI / params[1];
    mo.d[1] = params[0] * std::sin(w * t);
    mo.v[1] = params[0] * w * std::cos(w * t);
  }
  for (int c = 0; c < 3; ++c) {
    mo.dh[c] = (float)mo.d[c];
    mo.dl[c] = (float)(mo.d[c] - (double)mo.dh[c]);
  }
  return mo;
}

// Interpolation (+ force); with X0, also the L2 motion of `kind` at time t
// (X and Ud written to Xout, Udout).
template <typename T>
cudaError_t launch_interp(const ibm_plan_s *p, int n, const T *X, const T *u, const T *v, const T *w,
                          const T *du, const T *dv, const T *dw, T *U, const T *Ud, double inv_dt, T *F,
                          const T *X0, T *Xout, T *Udout, int kind, const double *params, double t,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const IbmGrid g = ibm_grid(p);
  const RigidMotion mo = X0 ? rigid_motion(kind, params, t) : RigidMotion{};
  const int tb = ceil_div(3 * n, kMarkerThreads);
  if (p->delta == IBM_DELTA_PESKIN4)
    IBM_KTRY(launch_pdl(k_interp<T, 4>, tb, kMarkerThreads, 0, st, g, n, X, u, v, w, du, dv, dw, U, Ud, (T)inv_dt,
                        F, X0, Xout, Udout, mo));
  else
    IBM_KTRY(launch_pdl(k_interp<T, 3>, tb, kMarkerThreads, 0, st, g, n, X, u, v, w, du, dv, dw, U, Ud, (T)inv_dt,
                        F, X0, Xout, Udout, mo));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const ibm_plan_s *p, int n, const T *X, const T *F, const T *dV, T *fu, T *fv, T *fw,
                          double scale, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const IbmGrid g = ibm_grid(p);
  const int tb = ceil_div(3 * n, 256);
  if (p->delta == IBM_DELTA_PESKIN4)
    IBM_KTRY(launch_pdl(k_spread<T, 4>, tb, 256, 0, st, g, n, X, F, dV, fu, fv, fw, (T)scale));
  else
    IBM_KTRY(launch_pdl(k_spread<T, 3>, tb, 256, 0, st, g, n, X, F, dV, fu, fv, fw, (T)scale));
  return cudaGetLastError();
}


template cudaError_t launch_interp<float>(const ibm_plan_s *, int, const float *, const float *, const float *,
                                          const float *, const float *, const float *, const float *, float *,
                                          const float *, double, float *, const float *, float *, float *, int,
                                          const double *, double, cudaStream_t);
template cudaError_t launch_interp<double>(const ibm_plan_s *, int, const double *, const double *,
                                           const double *, const double *, const double *, const double *,
                                           const double *, double *, const double *, double, double *,
                                           const double *, double *, double *, int, const double *, double,
                                           cudaStream_t);
template cudaError_t launch_spread<float>(const ibm_plan_s *, int, const float *, const float *, const float *,
                                          float *, float *, float *, double, cudaStream_t);
template cudaError_t launch_spread<double>(const ibm_plan_s *, int, const double *, const double *,
                                           const double *, double *, double *, double *, double, cudaStream_t);

}  // namespace ibm

using namespace ibm;

extern "C" {

int ibm_interp(ibm_plan plan, int n, const void *X, const void *u, const void *v, const void *w, void *U,
               void *stream) {
  if (!plan || n < 0 || (n > 0 && (!X || !u || !v || !w || !U)))
    return set_error(IBM_ERR_ARG, "ibm_interp: bad argument");
  if (plan->bc != IBM_BC_PXZ_WALL_Y)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_interp: the delta stencils are built for the wall-bounded branch");
  if (n > (1 << 28)) return set_error(IBM_ERR_ARG, "ibm_interp: n too large");
  cudaError_t e;
  if (plan->precision == IBM_FP64)
    e = launch_interp<double>(plan, n, (const double *)X, (const double *)u, (const double *)v, (const double *)w,
                              nullptr, nullptr, nullptr, (double *)U, nullptr, 0.0, nullptr, nullptr, nullptr, nullptr, 0,
                              nullptr, 0.0, (cudaStream_t)stream);
  else
    e = launch_interp<float>(plan, n, (const float *)X, (const float *)u, (const float *)v, (const float *)w,
                             nullptr, nullptr, nullptr, (float *)U, nullptr, 0.0, nullptr, nullptr, nullptr, nullptr, 0,
                             nullptr, 0.0, (cudaStream_t)stream);
  return e == cudaSuccess ? IBM_OK : cuda_error(e, "ibm_interp");
}

int ibm_spread(ibm_plan plan, int n, const void *X, const void *F, const void *dV, void *fu, void *fv, void *fw,
               void *stream) {
  if (!plan || n < 0 || (n > 0 && (!X || !F || !dV || !fu || !fv || !fw)))
    return set_error(IBM_ERR_ARG, "ibm_spread: bad argument");
  if (plan->bc != IBM_BC_PXZ_WALL_Y)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_spread: the delta stencils are built for the wall-bounded branch");
  if (n > (1 << 28)) return set_error(IBM_ERR_ARG, "ibm_spread: n too large");
  cudaError_t e;
  if (plan->precision == IBM_FP64)
    e = launch_spread<double>(plan, n, (const double *)X, (const double *)F, (const double *)dV, (double *)fu,
                              (double *)fv, (double *)fw, 1.0, (cudaStream_t)stream);
  else
    e = launch_spread<float>(plan, n, (const float *)X, (const float *)F, (const float *)dV, (float *)fu,
                             (float *)fv, (float *)fw, 1.0, (cudaStream_t)stream);
  return e == cudaSuccess ? IBM_OK : cuda_error(e, "ibm_spread");
}

}  // extern "C"
