// stencil.cuh -- the FP32 7-point residual at four consecutive x points,
// shared by the residual pass (stencil.cu) and the fused residual + x-rows
// pass of the slab solve (slab.cu).
#pragma once

#include "internal.h"

namespace ibm {

enum { BC_NEUMANN = 0, BC_CELL_DIRICHLET = 1, BC_FACE_DIRICHLET = 2, BC_PERIODIC = 3 };

struct ffc { float hi, lo; };
inline ffc split_ff(double v) {
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
// D_a = (x(+1) - x0) + (x(-1) - x0) the second difference along axis a.
// The second differences are where a plain FP32 stencil loses the residual:
// summed as x(+1) + x(-1) - 2 x0, O(|x|) values cancel to O(h^2 |x''|).  As
// differences from the centre value they are exact wherever the neighbours
// lie within a factor 2 of it (Sterbenz), i.e. everywhere a field is smooth
// on the grid scale, and only their sum is rounded, relative to D itself;
// where a field is rough, or crosses zero, the differences' rounding is
// O(eps |b|) and O(eps |x'| / h) respectively.  Every other term is O(|b|)
// and is summed in FP32 (K_a as its FP64 value split into hi + lo, the small
// products first): a few FP32 roundings of |b|, against a residual of an
// FP32 solution that is 1e-5 .. 1e-3 of |b| (its rounding errors are
// grid-scale, which L_h amplifies by ~1/h^2).  The correction is accurate to
// about 1 % and the refined solution reaches the FP32 rounding of its
// storage.
template <bool SIGMA>
__device__ __forceinline__ float residual_point(const ResidualArgs &A, float bv, float2 m, float x0, float xe, float xw,
                                                float xn, float xs, float xu, float xd, float &bt) {
  const float Dx = (xe - x0) + (xw - x0);
  const float Dz = (xn - x0) + (xs - x0);
  const float Dy = (xu - x0) + (xd - x0);
  const float bm = (bv - m.x) - m.y;
  bt = bm;
  float E = A.kx.lo * Dx;
  E = fmaf(A.kz.lo, Dz, E);
  E = fmaf(A.ky.lo, Dy, E);
  float S = SIGMA ? fmaf(-A.sigma, x0, bm) : bm;
  S = fmaf(A.kx.hi, Dx, S);
  S = fmaf(A.kz.hi, Dz, S);
  S = fmaf(A.ky.hi, Dy, S);
  return S + E;
}

// residual_point at two points at once with paired FP32 instructions
// (FADD2 / FMUL2 / FFMA2 on sm_100 and later): the same operations in the
// same order, each rounded once per lane, so the values equal
// residual_point's; a - b is fma(b, -1, a).
template <bool SIGMA>
__device__ __forceinline__ float2 residual_pair(const ResidualArgs &A, float2 bv, float2 m, float2 x0, float2 xe,
                                                float2 xw, float2 xn, float2 xs, float2 xu, float2 xd) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 Dx = __fadd2_rn(__ffma2_rn(x0, m1, xe), __ffma2_rn(x0, m1, xw));
  const float2 Dz = __fadd2_rn(__ffma2_rn(x0, m1, xn), __ffma2_rn(x0, m1, xs));
  const float2 Dy = __fadd2_rn(__ffma2_rn(x0, m1, xu), __ffma2_rn(x0, m1, xd));
  const float2 bm = __ffma2_rn(make_float2(m.y, m.y), m1, __ffma2_rn(make_float2(m.x, m.x), m1, bv));
  float2 E = __fmul2_rn(make_float2(A.kx.lo, A.kx.lo), Dx);
  E = __ffma2_rn(make_float2(A.kz.lo, A.kz.lo), Dz, E);
  E = __ffma2_rn(make_float2(A.ky.lo, A.ky.lo), Dy, E);
  float2 S = SIGMA ? __ffma2_rn(make_float2(-A.sigma, -A.sigma), x0, bm) : bm;
  S = __ffma2_rn(make_float2(A.kx.hi, A.kx.hi), Dx, S);
  S = __ffma2_rn(make_float2(A.kz.hi, A.kz.hi), Dz, S);
  S = __ffma2_rn(make_float2(A.ky.hi, A.ky.hi), Dy, S);
  return __fadd2_rn(S, E);
}

inline ResidualArgs make_args(int nx, int ny, int nz, const StencilCoef &c, const double *boff) {
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

// r at the four points (x = i0 .. i0 + 3, row k along z, plane j along y) of
// the wall kind BC, and the compatible right-hand side b - m there (bt, for
// the norms).  nx % 4 == 0 and 16-byte aligned fields: every row access is
// a float4; the x neighbours of the four come from the same float4 plus two
// scalars.
template <int BC, bool SIGMA>
__device__ __forceinline__ float4 residual4(const ResidualArgs &A, const float *__restrict__ b,
                                            const float *__restrict__ x, int j, int k, int i0, float2 m,
                                            float4 &bt) {
  const size_t pl = (size_t)A.nx * A.nz;
  const size_t at = (size_t)j * pl + (size_t)k * A.nx + i0;
  float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
  bt = res;
  if (BC == BC_FACE_DIRICHLET && j == 0) return res;
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
  res.x = residual_point<SIGMA>(A, bv.x, m, x0.x, x0.y, xW, xn.x, xs.x, xu.x, xd.x, bt.x);
  res.y = residual_point<SIGMA>(A, bv.y, m, x0.y, x0.z, x0.x, xn.y, xs.y, xu.y, xd.y, bt.y);
  res.z = residual_point<SIGMA>(A, bv.z, m, x0.z, x0.w, x0.y, xn.z, xs.z, xu.z, xd.z, bt.z);
  res.w = residual_point<SIGMA>(A, bv.w, m, x0.w, xE, x0.z, xn.w, xs.w, xu.w, xd.w, bt.w);
  return res;
}

// The same four points for a block of consecutive rows of one y plane
// (the wall kinds Neumann and cell Dirichlet only), with the addressing
// reduced to 32-bit offsets from the block's first row: xc, bc point at x, b
// there, xlo / xhi at x one plane below / above (NULL at a wall: the ghost
// value), off = (row - first row) nx + i0, k the row's z index.
template <int BC, bool SIGMA>
__device__ __forceinline__ float4 residual4_rows(const ResidualArgs &A, const float *__restrict__ bc,
                                                 const float *__restrict__ xc, const float *__restrict__ xlo,
                                                 const float *__restrict__ xhi, int off, int i0, int k, float2 m,
                                                 float4 &bt) {
  static_assert(BC == BC_NEUMANN || BC == BC_CELL_DIRICHLET, "wall kinds with ghost values");
  const int nx = A.nx;
  const float4 x0 = *reinterpret_cast<const float4 *>(xc + off);
  const float xW = xc[off + (i0 == 0 ? nx - 1 : -1)];
  const float xE = xc[off + (i0 + 4 == nx ? 4 - nx : 4)];
  const int dn = k + 1 == A.nz ? -(A.nz - 1) * nx : nx;
  const int ds = k == 0 ? (A.nz - 1) * nx : -nx;
  const float4 xn = *reinterpret_cast<const float4 *>(xc + off + dn);
  const float4 xs = *reinterpret_cast<const float4 *>(xc + off + ds);
  const float gs = BC == BC_NEUMANN ? 1.0f : -1.0f;
  const float4 xd = xlo ? *reinterpret_cast<const float4 *>(xlo + off)
                        : make_float4(gs * x0.x, gs * x0.y, gs * x0.z, gs * x0.w);
  const float4 xu = xhi ? *reinterpret_cast<const float4 *>(xhi + off)
                        : make_float4(gs * x0.x, gs * x0.y, gs * x0.z, gs * x0.w);
  const float4 bv = *reinterpret_cast<const float4 *>(bc + off);
  float4 res;
  res.x = residual_point<SIGMA>(A, bv.x, m, x0.x, x0.y, xW, xn.x, xs.x, xu.x, xd.x, bt.x);
  res.y = residual_point<SIGMA>(A, bv.y, m, x0.y, x0.z, x0.x, xn.y, xs.y, xu.y, xd.y, bt.y);
  res.z = residual_point<SIGMA>(A, bv.z, m, x0.z, x0.w, x0.y, xn.z, xs.z, xu.z, xd.z, bt.z);
  res.w = residual_point<SIGMA>(A, bv.w, m, x0.w, xE, x0.z, xn.w, xs.w, xu.w, xd.w, bt.w);
  return res;
}

// The four points' shares of the norm sums (r^2, b^2, r, b).
__device__ __forceinline__ void residual4_norms(float4 res, float4 bt, double &r2, double &b2, double &r1,
                                                double &b1) {
  r2 += (double)res.x * res.x + (double)res.y * res.y + (double)res.z * res.z + (double)res.w * res.w;
  b2 += (double)bt.x * bt.x + (double)bt.y * bt.y + (double)bt.z * bt.z + (double)bt.w * bt.w;
  r1 += (double)res.x + res.y + res.z + res.w;
  b1 += (double)bt.x + bt.y + bt.z + bt.w;
}

}  // namespace ibm
