// ibm_kernels.cu -- Lagrangian operations of the immersed boundary (Sec. 2.3.2).
//
// Interpolation (Eq. 2b) and spreading (Eq. 2d) with a regularised delta
// delta_h(x - X) = phi((x-X)/hx) phi((y-Y)/hy) phi((z-Z)/hz) / (hx hy hz).
// The paper cites Peskin and Roma et al. without printing phi; ROMA3 is the
// three-point kernel of Roma, Peskin & Berger (1999), PESKIN4 the four-point
// kernel of Peskin (2002).  Each velocity component lives on its own
// staggered sub-grid (origin in grid units: u (0,1/2,1/2), v (1/2,0,1/2),
// w (1/2,1/2,0)); x and z wrap periodically.  Along y the support of an
// S-point kernel reaches S/2 cells from the marker; a marker closer than
// that to a wall (Y < (S/2) hy or Y > Ly - (S/2) hy) would need values
// beyond the wall and is rejected: it is neither interpolated (its U and F
// are 0) nor spread, and the plan's error word records it (kErrWall and a
// count), which ibm_plan_check reports as IBM_ERR_ARG.  Every support point
// of an accepted marker is a stored unknown (v's wall face 0 included:
// accepted markers give it zero weight).
//
// One thread per (marker, component).  The stencil origin and offset are
// computed in FP64 on the FP64 path and in float-float on the FP32 path, so
// that the weights see the marker position without the FP32 rounding of
// X/h; the weights and sums run in the plan precision.  Spreading
// accumulates with global atomics as in the paper's L1 kernel (Sec. 2.3.2).
#include <algorithm>
#include <climits>
#include <cmath>

#include "plan.h"
#include "tma.cuh"

namespace ibm {

struct IbmGrid {
  int nx, ny, nz;
  double inv_h[3];
  float ih_hi[3], ih_lo[3];  // 1/h as float-float for the FP32 path
  double vol_inv;            // 1 / (hx hy hz)
  int *err;                  // the plan's error word (flags, rejected-marker count)
};

// The wall rule: Y at least S/2 cells from both walls.  FP64: plain
// doubles.  FP32: Y / hy as a float-float (the error-free product used for
// the stencil origin), so the decision does not see the rounding of Y / hy.
template <int S> __device__ __forceinline__ bool clear_of_walls(const IbmGrid &g, double Y) {
  const double s = Y * g.inv_h[1], r = 0.5 * S;
  return s >= r && s <= (double)g.ny - r;
}
template <int S> __device__ __forceinline__ bool clear_of_walls(const IbmGrid &g, float Y) {
  const ff p = two_prod(Y, g.ih_hi[1]);
  const float lo = fmaf(Y, g.ih_lo[1], p.lo);
  const float r = 0.5f * S;
  return (p.hi - r) + lo >= 0.f && (((float)g.ny - r) - p.hi) - lo >= 0.f;
}
__device__ __forceinline__ void report_wall(const IbmGrid &g) {
  atomicOr(g.err, kErrWall);
  atomicAdd(g.err + 1, 1);
}

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
  if (!clear_of_walls<S>(g, my)) {  // the wall rule: no interpolation, no force
    if (c == 0) report_wall(g);
    if (U) U[t] = (T)0;
    if (F) F[t] = (T)0;
    return;
  }
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
  if (!clear_of_walls<S>(g, X[3 * m + 1])) {  // the wall rule: not spread
    if (c == 0) report_wall(g);
    return;
  }
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

// Spreading with shared-memory pre-aggregation (the default atomic path).
// Markers that are close in index are usually close in space (a surface
// mesh, a lattice, a Fibonacci sphere's latitude bands), so the 256
// entries of a CTA touch a small box of grid points while many markers hit
// the same points.  The CTA finds the bounding box of its stencils (in
// unwrapped index space, all three components together); if the box fits
// the shared budget, the stencils accumulate there with shared-memory
// atomics and each non-zero box point is added to the field with one
// global atomic (x and z wrapped, points beyond the walls dropped as in
// k_spread).  Otherwise the CTA falls back to k_spread's direct global
// atomics.  Same sums in another order (FP32 atomics are unordered anyway).
// Measured on GB300 (FP32, a Fibonacci sphere of radius 0.25 at 128^3): 20k
// markers 21.2 us against 16.7 us for direct atomics (little contention:
// the extra phases cost more than they save); 100k markers 38.3 us against
// 81.6 us.  IBM_SPREAD_ATOMIC therefore takes this kernel from
// kSpreadBoxMinMarkers markers on.
constexpr int kSpreadBoxMinMarkers = 40000;
constexpr int kSpreadBoxBytes = 40 * 1024;  // within the default 48 KB limit with the static part

template <typename T, int S>
__global__ void __launch_bounds__(256)
k_spread_box(IbmGrid g, int n, const T *__restrict__ X, const T *__restrict__ F, const T *__restrict__ dV, T *fu,
             T *fv, T *fw, T scale) {
  extern __shared__ __align__(16) unsigned char box_raw[];
  T *box = reinterpret_cast<T *>(box_raw);
  __shared__ int red[6][8];
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = t < 3 * n ? t / 3 : 0, c = t < 3 * n ? t - 3 * m : 0;
  bool valid = t < 3 * n;
  if (valid && !clear_of_walls<S>(g, X[3 * m + 1])) {  // the wall rule: not spread
    if (c == 0) report_wall(g);
    valid = false;
  }
  int bx = 0, by = 0, bz = 0;
  T fx = 0, fy = 0, fz = 0, amp = 0;
  if (valid) {
    stencil_origin<T, S>(g, c, X[3 * m], X[3 * m + 1], X[3 * m + 2], bx, by, bz, fx, fy, fz);
    amp = scale * F[t] * dV[m] * (T)g.vol_inv;
  }
  // bounding box of the CTA's stencil origins
  int v[6] = {valid ? bx : INT_MAX, valid ? by : INT_MAX, valid ? bz : INT_MAX,
              valid ? -bx : INT_MAX, valid ? -by : INT_MAX, valid ? -bz : INT_MAX};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    v[q] = __reduce_min_sync(0xffffffffu, v[q]);
    if (lane == 0) red[q][warp] = v[q];
  }
  __syncthreads();
  int lo[3], dim[3];
  bool any = false;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    int mn = INT_MAX, mxn = INT_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      mn = min(mn, red[q][w]);
      mxn = min(mxn, red[q + 3][w]);
    }
    any = mn != INT_MAX;  // the same for every axis and every thread
    lo[q] = any ? mn : 0;
    dim[q] = any ? -mxn - mn + S : 0;  // (max - min) + S points along this axis
  }
  if (!any) return;  // every entry of the CTA was rejected by the wall rule
  const long vol = (long)dim[0] * dim[1] * dim[2];
  const bool use_box = vol > 0 && 3 * vol * (long)sizeof(T) <= kSpreadBoxBytes && dim[0] <= g.nx && dim[2] <= g.nz;
  T wx[S], wz[S];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    wx[q] = S == 3 ? phi_roma3<T>(fx - (T)q) : phi_peskin4<T>(fx - (T)q);
    wz[q] = S == 3 ? phi_roma3<T>(fz - (T)q) : phi_peskin4<T>(fz - (T)q);
  }
  const int jlo = c == 1 ? 1 : 0;
  if (!use_box) {
    if (!valid) return;
    T *f = c == 0 ? fu : c == 1 ? fv : fw;
    int ix[S], kz[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
      ix[q] = wrap(bx + q, g.nx);
      kz[q] = wrap(bz + q, g.nz);
    }
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
    return;
  }
  const int nbox = 3 * (int)vol;
  for (int e = threadIdx.x; e < nbox; e += blockDim.x) box[e] = (T)0;
  __syncthreads();
  if (valid) {
    T *bc = box + c * (int)vol;
    const int ox = bx - lo[0], oy = by - lo[1], oz = bz - lo[2];
#pragma unroll
    for (int qy = 0; qy < S; ++qy) {
      const T wy = S == 3 ? phi_roma3<T>(fy - (T)qy) : phi_peskin4<T>(fy - (T)qy);
#pragma unroll
      for (int qz = 0; qz < S; ++qz) {
        T *rowp = bc + ((oy + qy) * dim[2] + (oz + qz)) * dim[0] + ox;
        const T a = amp * wy * wz[qz];
#pragma unroll
        for (int qx = 0; qx < S; ++qx) atomicAdd(rowp + qx, a * wx[qx]);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nbox; e += blockDim.x) {
    const T val = box[e];
    if (val == (T)0) continue;
    const int cc = e / (int)vol;
    int r = e - cc * (int)vol;
    const int dy = r / (dim[2] * dim[0]);
    r -= dy * dim[2] * dim[0];
    const int dz = r / dim[0], dx = r - dz * dim[0];
    const int j = lo[1] + dy;
    if (j < (cc == 1 ? 1 : 0) || j > g.ny - 1) continue;
    const int i = wrap(lo[0] + dx, g.nx), k = wrap(lo[2] + dz, g.nz);
    T *f = cc == 0 ? fu : cc == 1 ? fv : fw;
    atomicAdd(f + ((size_t)j * g.nz + k) * g.nx + i, val);
  }
}

// ---------------------------------------------------------------------------
// Deterministic spreading by Eulerian gather (IBM_SPREAD_GATHER).
//
// Every (marker, component) entry t = 3 m + c gets a stencil record (origin
// b, offsets f, amplitude F dV / (hx hy hz)).  Entries are grouped by the
// cell of their origin in component c's grid (y shifted by 2 so that origins
// below the first row have a cell too): a counting sort into 4^3 bricks,
// then, per non-empty brick, a counting sort into its 64 cells, and each
// cell's entries ordered by t.  A grid point is covered exactly by the
// entries whose origin lies in one of the S^3 cells at most S - 1 below it
// along each axis; it visits those cells in a fixed order and their entries
// in t order, so its sum has the same order on every run.  Only target
// bricks (those some stencil touches) are visited.
// ---------------------------------------------------------------------------
constexpr int kBrick = 4;
constexpr int kCells = kBrick * kBrick * kBrick;

template <typename T> struct StencilRec {
  int bx, by, bz;  // origin (bx, bz wrapped into the periodic range)
  T fx, fy, fz, amp;
};

struct BrickGeom {
  int nbx, nby, nbz, nb;  // bricks per axis and per component (nb = nbx nby nbz)
};

__device__ __forceinline__ int brick_of(const BrickGeom &bg, int c, int xb, int yb, int zb) {
  return ((c * bg.nbz + zb) * bg.nby + yb) * bg.nbx + xb;
}

// Cell (wrapped x, z; y + 2 clamped, so that any origin, even one of a marker
// outside the walls, has one) of a stencil origin: its brick and its index
// in the brick.
__device__ __forceinline__ void origin_cell(const IbmGrid &g, const BrickGeom &bg, int c, int bx, int by, int bz,
                                            int &brick, int &cell) {
  const int x = wrap(bx, g.nx), z = wrap(bz, g.nz), y = min(max(by + 2, 0), bg.nby * kBrick - 1);
  brick = brick_of(bg, c, x / kBrick, y / kBrick, z / kBrick);
  cell = ((z % kBrick) * kBrick + y % kBrick) * kBrick + x % kBrick;
}

// Block-wide exclusive scan of one int per thread.
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const int x = lane < nw ? warp_sums[lane] : 0;
    int xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += u;
    }
    if (lane < nw) warp_sums[lane] = xi - x;
  }
  __syncthreads();
  const int r = warp_sums[w] + incl - v;
  __syncthreads();
  return r;
}

template <typename T, int S>
__global__ void __launch_bounds__(256)
k_gather_prep(IbmGrid g, BrickGeom bg, int n, const T *__restrict__ X, const T *__restrict__ F,
              const T *__restrict__ dV, T scale, StencilRec<T> *__restrict__ rec, int *__restrict__ count,
              int *__restrict__ target, int *__restrict__ tlist, int *__restrict__ blist, int *__restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int m = t / 3, c = t - 3 * m;
  StencilRec<T> r;
  stencil_origin<T, S>(g, c, X[3 * m], X[3 * m + 1], X[3 * m + 2], r.bx, r.by, r.bz, r.fx, r.fy, r.fz);
  r.amp = scale * F[t] * dV[m] * (T)g.vol_inv;
  if (!clear_of_walls<S>(g, X[3 * m + 1])) {  // the wall rule: a record that adds nothing
    if (c == 0) report_wall(g);
    r.amp = (T)0;
  }
  const int bx_raw = r.bx, bz_raw = r.bz;
  r.bx = wrap(r.bx, g.nx);  // records keep the periodic origins wrapped
  r.bz = wrap(r.bz, g.nz);
  rec[t] = r;
  int brick, cell;
  origin_cell(g, bg, c, r.bx, r.by, r.bz, brick, cell);
  // the first entry of a brick lists it (list order is immaterial: every
  // brick's range and every point's sum are formed in a fixed order later)
  if (atomicAdd(count + brick, 1) == 0) blist[atomicAdd(cnt + 1, 1)] = brick;
  // bricks the stencil touches (points b .. b + S - 1 per axis)
  const int xa = r.bx / kBrick, xe = wrap(bx_raw + S - 1, g.nx) / kBrick;
  const int za = r.bz / kBrick, ze = wrap(bz_raw + S - 1, g.nz) / kBrick;
  const int ya = min(max(r.by + 2, 0), bg.nby * kBrick - 1) / kBrick;
  const int ye = min(max(r.by + 2 + S - 1, 0), bg.nby * kBrick - 1) / kBrick;
  const int xs[2] = {xa, xe}, ys[2] = {ya, ye}, zs[2] = {za, ze};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int tb = brick_of(bg, c, xs[d], ys[b], zs[a]);
        if (target[tb] == 0 && atomicExch(target + tb, 1) == 0) tlist[atomicAdd(cnt, 1)] = tb;
      }
}

// One CTA of 1024 threads: the entry ranges of the listed non-empty bricks
// (offq[q] .. offq[q + 1] for brick blist[q]; rank[blist[q]] = q).
__global__ void __launch_bounds__(1024)
k_gather_ranges(const int *__restrict__ count, const int *__restrict__ blist, const int *__restrict__ cnt,
                int *__restrict__ offq, int *__restrict__ rank) {
  __shared__ int ws[32];
  __shared__ int tot;
  const int nb = cnt[1];
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int q = base + threadIdx.x;
    const int v = q < nb ? count[blist[q]] : 0;
    const int e = block_excl_scan(v, ws) + carry;
    if (q < nb) { offq[q] = e; rank[blist[q]] = q; }
    if (threadIdx.x == blockDim.x - 1) tot = e + v;
    __syncthreads();
    carry = tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) offq[nb] = carry;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gather_scatter(IbmGrid g, BrickGeom bg, int n, const StencilRec<T> *__restrict__ rec, const int *__restrict__ offq,
                 const int *__restrict__ rank, int *__restrict__ fill, int *__restrict__ entry) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const StencilRec<T> r = rec[t];
  int brick, cell;
  origin_cell(g, bg, t % 3, r.bx, r.by, r.bz, brick, cell);
  entry[offq[rank[brick]] + atomicAdd(fill + brick, 1)] = t;
}

// Per listed brick (one CTA each, grid-stride): its entries by cell (cell
// offsets, relative to the brick's range, in coff[q * 65 ..]) and, within a
// cell, in ascending t, as their records in srec.  A brick's entries are
// grouped in shared memory up to kSortCap of them, in global memory
// (sorted[]) beyond.
constexpr int kSortCap = 6144;

template <typename T>
__global__ void __launch_bounds__(256)
k_gather_cells(IbmGrid g, BrickGeom bg, const StencilRec<T> *__restrict__ rec, const int *__restrict__ offq,
               const int *__restrict__ blist, const int *__restrict__ cnt, const int *__restrict__ entry,
               int *__restrict__ sorted, int *__restrict__ coff, StencilRec<T> *__restrict__ srec) {
  __shared__ int hist[kCells], start[kCells + 1], fillc[kCells];
  __shared__ int buf[kSortCap];
  const int nb = cnt[1];
  for (int q = blockIdx.x; q < nb; q += gridDim.x) {
    const int b = blist[q];
    const int lo = offq[q], hi = offq[q + 1];
    const int c = b / bg.nb;
    int *dst = hi - lo <= kSortCap ? buf : sorted + lo;
    if (threadIdx.x < kCells) { hist[threadIdx.x] = 0; fillc[threadIdx.x] = 0; }
    __syncthreads();
    for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const StencilRec<T> r = rec[entry[e]];
      int brick, cell;
      origin_cell(g, bg, c, r.bx, r.by, r.bz, brick, cell);
      atomicAdd(hist + cell, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int k = 0; k < kCells; ++k) { start[k] = acc; acc += hist[k]; }
      start[kCells] = acc;
    }
    __syncthreads();
    if (threadIdx.x <= kCells) coff[(size_t)q * (kCells + 1) + threadIdx.x] = start[threadIdx.x];
    for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const int t = entry[e];
      const StencilRec<T> r = rec[t];
      int brick, cell;
      origin_cell(g, bg, c, r.bx, r.by, r.bz, brick, cell);
      dst[start[cell] + atomicAdd(fillc + cell, 1)] = t;
    }
    __syncthreads();
    // t order within each cell: an entry's place is the number of entries of
    // its cell with a smaller t (t values are distinct)
    for (int e = threadIdx.x; e < hi - lo; e += blockDim.x) {
      const int t = dst[e];
      int cell = 0;
      while (start[cell + 1] <= e) ++cell;
      int rk = 0;
      for (int i = start[cell]; i < start[cell + 1]; ++i) rk += dst[i] < t ? 1 : 0;
      srec[lo + start[cell] + rk] = rec[t];
    }
    __syncthreads();
  }
}

// One CTA of 8 warps per target brick (grid-stride over the target list).
// The entry ranges of the (4 + S - 1)^3 origin cells its points can need are
// looked up once into shared memory; then a warp takes the brick's points in
// turn, and for each of a point's S^3 origin cells (fixed order) lane l takes
// the cell's entries l, l + 32, ...; the lanes' sums are added by a fixed
// butterfly: the same order on every run.
template <typename T, int S>
__global__ void __launch_bounds__(256)
k_gather(IbmGrid g, BrickGeom bg, const int *__restrict__ tlist, const int *__restrict__ cnt,
         const int *__restrict__ count, const int *__restrict__ offq, const int *__restrict__ rank,
         const int *__restrict__ coff, const StencilRec<T> *__restrict__ srec, T *fu, T *fv, T *fw) {
  constexpr int E = kBrick + S - 1;  // origin cells per axis
  __shared__ int rlo[E * E * E], rhi[E * E * E];
  const int nt = cnt[0];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = blockIdx.x; q < nt; q += gridDim.x) {
    const int bid = tlist[q];
    const int c = bid / bg.nb;
    int rem = bid - c * bg.nb;
    const int zb = rem / (bg.nby * bg.nbx);
    rem -= zb * bg.nby * bg.nbx;
    const int yb = rem / bg.nbx, xb = rem - yb * bg.nbx;
    const int i0 = xb * kBrick - (S - 1), k0 = zb * kBrick - (S - 1), j0 = yb * kBrick - 2 - (S - 1);
    for (int u = threadIdx.x; u < E * E * E; u += blockDim.x) {
      const int ox = u % E, oy = (u / E) % E, oz = u / (E * E);
      int brick, cell;
      origin_cell(g, bg, c, i0 + ox, j0 + oy, k0 + oz, brick, cell);
      int a = 0, z = 0;
      if (count[brick] != 0) {
        const int qq = rank[brick];
        const int base = offq[qq];
        const int *co = coff + (size_t)qq * (kCells + 1);
        a = base + co[cell];
        z = base + co[cell + 1];
      }
      rlo[u] = a;
      rhi[u] = z;
    }
    __syncthreads();
    const int jlo = c == 1 ? 1 : 0;
    T *f = c == 0 ? fu : c == 1 ? fv : fw;
    for (int pt = w; pt < kCells; pt += 8) {
      const int px = pt % kBrick, py = (pt / kBrick) % kBrick, pz = pt / (kBrick * kBrick);
      const int i = xb * kBrick + px, k = zb * kBrick + pz, j = yb * kBrick + py - 2;
      if (j < jlo || j > g.ny - 1) continue;  // warp-uniform
      T acc = (T)0;
      bool any = false;
      for (int qz = 0; qz < S; ++qz) {
        for (int qy = 0; qy < S; ++qy) {
          for (int qx = 0; qx < S; ++qx) {
            const int u = ((pz + S - 1 - qz) * E + (py + S - 1 - qy)) * E + (px + S - 1 - qx);
            const int bx = i - qx < 0 ? i - qx + g.nx : i - qx, by = j - qy;
            const int bz = k - qz < 0 ? k - qz + g.nz : k - qz;
            for (int e = rlo[u] + lane; e < rhi[u]; e += 32) {
              const StencilRec<T> r = srec[e];
              // the cell holds every origin that maps to it; keep the exact one
              if (r.bx != bx || r.by != by || r.bz != bz) continue;
              const T wx = S == 3 ? phi_roma3<T>(r.fx - (T)qx) : phi_peskin4<T>(r.fx - (T)qx);
              const T wy = S == 3 ? phi_roma3<T>(r.fy - (T)qy) : phi_peskin4<T>(r.fy - (T)qy);
              const T wz = S == 3 ? phi_roma3<T>(r.fz - (T)qz) : phi_peskin4<T>(r.fz - (T)qz);
              acc += r.amp * (wy * wz) * wx;
              any = true;
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (__any_sync(0xffffffffu, any) && lane == 0) f[((size_t)j * g.nz + k) * g.nx + i] += acc;
    }
    __syncthreads();  // the range tables are reused by the next brick
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
  g.err = p->derr;
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

// Workspace of the gather: ints count, fill, target, rank (len each), tlist,
// blist, offq (len + 1 each), cnt (2), entry, sorted (3 n each), coff
// (min(3 n, len) x 65); then the stencil records and the same in cell order
// (3 n each).
template <typename T>
static int spread_gather(ibm_plan_s *p, int n, const T *X, const T *F, const T *dV, T *fu, T *fv, T *fw,
                         double scale, cudaStream_t st) {
  const IbmGrid g = ibm_grid(p);
  BrickGeom bg;
  bg.nbx = ceil_div(p->nx, kBrick);
  bg.nby = ceil_div(p->ny + 4, kBrick);
  bg.nbz = ceil_div(p->nz, kBrick);
  bg.nb = bg.nbx * bg.nby * bg.nbz;
  const int len = 3 * bg.nb;
  const size_t ne = 3 * (size_t)n;
  const size_t nbrk = std::min(ne, (size_t)len);
  const size_t ints = 4 * (size_t)len + 3 * ((size_t)len + 1) + 2 + 2 * ne + nbrk * (kCells + 1);
  const size_t rec_off = (ints * sizeof(int) + 15) & ~(size_t)15;
  const size_t need = rec_off + 2 * ne * sizeof(StencilRec<T>);
  if (need > p->gcap) {
    if (p->gbuf) { cudaFree(p->gbuf); p->bytes -= p->gcap; p->gbuf = nullptr; p->gcap = 0; }
    cudaError_t e = cudaMalloc(&p->gbuf, need);
    if (e != cudaSuccess) { p->gbuf = nullptr; return set_error(IBM_ERR_OOM, "gather-spreading workspace"); }
    p->gcap = need;
    p->bytes += need;
  }
  int *count = static_cast<int *>(p->gbuf);
  int *fill = count + len, *target = fill + len, *rank = target + len;
  int *tlist = rank + len, *blist = tlist + len + 1, *offq = blist + len + 1, *cnt = offq + len + 1;
  int *entry = cnt + 2, *sorted = entry + ne, *coff = sorted + ne;
  StencilRec<T> *rec = reinterpret_cast<StencilRec<T> *>(static_cast<char *>(p->gbuf) + rec_off);
  StencilRec<T> *srec = rec + ne;
  IBM_CUDA_TRY(cudaMemsetAsync(count, 0, 3 * (size_t)len * sizeof(int), st));  // count, fill, target
  IBM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st));
  const int tb = ceil_div((int)ne, 256);
  if (p->delta == IBM_DELTA_PESKIN4)
    k_gather_prep<T, 4><<<tb, 256, 0, st>>>(g, bg, n, X, F, dV, (T)scale, rec, count, target, tlist, blist, cnt);
  else
    k_gather_prep<T, 3><<<tb, 256, 0, st>>>(g, bg, n, X, F, dV, (T)scale, rec, count, target, tlist, blist, cnt);
  k_gather_ranges<<<1, 1024, 0, st>>>(count, blist, cnt, offq, rank);
  k_gather_scatter<T><<<tb, 256, 0, st>>>(g, bg, n, rec, offq, rank, fill, entry);
  const int cgrid = (int)std::min(nbrk, (size_t)152 * 8);
  k_gather_cells<T><<<cgrid, 256, 0, st>>>(g, bg, rec, offq, blist, cnt, entry, sorted, coff, srec);
  const int grid = std::min(len, 152 * 8);
  if (p->delta == IBM_DELTA_PESKIN4)
    k_gather<T, 4><<<grid, 256, 0, st>>>(g, bg, tlist, cnt, count, offq, rank, coff, srec, fu, fv, fw);
  else
    k_gather<T, 3><<<grid, 256, 0, st>>>(g, bg, tlist, cnt, count, offq, rank, coff, srec, fu, fv, fw);
  IBM_CUDA_TRY(cudaGetLastError());
  return IBM_OK;
}

template <typename T>
cudaError_t launch_spread(const ibm_plan_s *p, int n, const T *X, const T *F, const T *dV, T *fu, T *fv, T *fw,
                          double scale, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (p->spread == IBM_SPREAD_GATHER) {
    // the workspace may grow: the plan is single-stream, so it is not in use
    const int rc = spread_gather<T>(const_cast<ibm_plan_s *>(p), n, X, F, dV, fu, fv, fw, scale, st);
    return rc == IBM_OK ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  const IbmGrid g = ibm_grid(p);
  const int tb = ceil_div(3 * n, 256);
  if (p->spread == IBM_SPREAD_ATOMIC_DIRECT || n < kSpreadBoxMinMarkers) {
    if (p->delta == IBM_DELTA_PESKIN4)
      IBM_KTRY(launch_pdl(k_spread<T, 4>, tb, 256, 0, st, g, n, X, F, dV, fu, fv, fw, (T)scale));
    else
      IBM_KTRY(launch_pdl(k_spread<T, 3>, tb, 256, 0, st, g, n, X, F, dV, fu, fv, fw, (T)scale));
    return cudaGetLastError();
  }
  if (p->delta == IBM_DELTA_PESKIN4)
    IBM_KTRY(launch_pdl(k_spread_box<T, 4>, tb, 256, (size_t)kSpreadBoxBytes, st, g, n, X, F, dV, fu, fv, fw,
                        (T)scale));
  else
    IBM_KTRY(launch_pdl(k_spread_box<T, 3>, tb, 256, (size_t)kSpreadBoxBytes, st, g, n, X, F, dV, fu, fv, fw,
                        (T)scale));
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
