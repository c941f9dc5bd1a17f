// seg.cuh -- the per-segment steps of the segmented two-ended pencil sweep
// (pencil.cu k_pencil_seg, slab.cu k_slab): one thread owns one pencil's S
// consecutive rows of a half sweep, counted from the wall (k = k0 .. k0 +
// len - 1), in registers.  With M = tridiag(-a, 2a + g, -a) in excess form
// (pivot p_k = a + e_k, e_k = g + a q_{k-1}, q_k = e_k / p_k, w_k = a / p_k):
//   forward     y_k = sgn f_k / p_k + w_k y_{k-1}   (from a zero carry)
//   middle      carry c = y before the segment folded in, then the local back
//               substitution x_k = y_k + w_k x_{k+1} from a zero carry
//   store       carry x after the segment folded in, rows written out.
// The pivot at the segment's first row comes in closed form from the fixed
// points of the Moebius map e -> g + a e / (a + e) (seg_pivots).  WST is the
// stride (in elements) between consecutive rows of the thread's w entries.
#pragma once

#include "internal.h"
#include "tma.cuh"

namespace ibm {

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return rcp_approx(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_excl_scan(double v, int lane) {
  double s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += t;
  }
  return s - v;
}

// FP64 zero-mode pencil, run by one full warp of a CTA of its own (the last
// CTA of the pencil grid) concurrently with the other pencils.  Input
// f_j = Re S[j][0][0] (zrhs, written by the forward transform); output
// zsol[j] (read by the inverse transform).  zs is shared scratch of ny doubles.
// zrhs, zsol and zs may be one array: each lane reads and writes only its
// own rows, zrhs before zs and zs before zsol.
__device__ __forceinline__ void zero_mode_fp64(const double *zrhs, double *zsol, double *zs, int ny,
                               double inv_ny, double hy2, double inv_nxnz, double *mean_out) {
  const int lane = threadIdx.x & 31;
  const int c = (ny + 31) / 32;
  const int lo = min(ny, lane * c), hi = min(ny, lo + c);
  double s = 0.0;
  for (int j = lo; j < hi; ++j) {
    const double v = zrhs[j];
    zs[j] = v;
    s += v;
  }
  const double mean = warp_sum(s) * inv_ny;
  if (lane == 0 && mean_out) {
    const double m = mean * inv_nxnz;
    mean_out[0] = m;
    // the same value as a float-float pair for FP32 consumers
    float2 f;
    f.x = (float)m;
    f.y = (float)(m - (double)f.x);
    *reinterpret_cast<float2 *>(mean_out + 1) = f;
  }
  // F_j = sum_{i <= j} (f_i - mean)
  double acc = 0.0;
  for (int j = lo; j < hi; ++j) { acc += zs[j] - mean; zs[j] = acc; }
  double off = warp_excl_scan(acc, lane);
  for (int j = lo; j < hi; ++j) zs[j] += off;
  __syncwarp();
  // x_j = hy^2 sum_{i < j} F_i   (x_0 = 0: the pin at the first interior point)
  double acc2 = 0.0;
  for (int j = lo; j < hi; ++j) { const double t = zs[j]; zs[j] = acc2; acc2 += t; }
  off = warp_excl_scan(acc2, lane);
  double s2 = 0.0;
  for (int j = lo; j < hi; ++j) { zs[j] = (zs[j] + off) * hy2; s2 += zs[j]; }
  const double m2 = warp_sum(s2) * inv_ny;
  for (int j = lo; j < hi; ++j) zsol[j] = zs[j] - m2;
}

// Closed-form pivot data at distance k0 from the wall: fixed points e+ > 0 >
// e- = -a g / e+, D = e+ - e-, z = (e0 - e+) / (e0 - e-) lambda^k0 with
// 1 - lambda = (a g + e+^2) / (e+ (a + e+)) (free of cancellation); the
// singular zero pencil (g = 0) gets ep = D = z = 0.  ok: |z| is below a
// sixteenth of the unit roundoff (the converged pivot e+ holds from k0 on).
template <typename T>
__device__ __forceinline__ bool seg_pivots(T a, T g, T e0, int k0, T &ep, T &D, T &z) {
  const bool zero = g == (T)0;
  const T gg = zero ? (T)1 : g;
  ep = (T)0.5 * (gg + sqrt(fma(gg, gg, (T)4 * a * gg)));
  const T emn = a * gg / ep;  // -e-
  D = ep + emn;
  const T mu = fma(ep, ep, a * gg) / (ep * (a + ep));
  z = (e0 - ep) / (e0 + emn);
  if constexpr (sizeof(T) == 4) {
    const T lam = fmaxf(log1pf(-mu), -80.0f);  // log lambda
    z *= expf((T)k0 * lam);
  } else {
    const T lam = (T)1 - mu;
    T lp = (T)1, base = lam;
    for (int kk = k0; kk; kk >>= 1) {
      if (kk & 1) lp *= base;
      base *= base;
    }
    z *= lp;
  }
  if (zero) { ep = (T)0; D = (T)0; z = (T)0; }
  return fabs(z) < (sizeof(T) == 4 ? (T)0x1p-28 : (T)0x1p-56);
}

// Per-warp sweep variants: FULL (all S rows of the segment are unknowns, no
// row guards) and CW (converged pivots: constant r and w).  Rows u >= len of a
// partial segment are pass-through (r = 0, w = 1) and read as zero.
template <typename T, int S, bool FULL, bool CW, int WST = 32>
__device__ __forceinline__ void seg_forward(cplx<T> (&v)[S], int len, int k0, T a, T g, T e0, T sgn, T ep, T D, T z,
                                            T *wc, cplx<T> &y, T &prod, T &qlast) {
  y = mk<T>(0, 0);
  prod = (T)1;
  qlast = (T)0;
  if (CW) {
    const T r = rcp<T>(a + ep), w = a * r, rs = sgn * r;
#pragma unroll
    for (int u = 0; u < S; ++u) {
      y.x = fma(w, y.x, rs * v[u].x);
      y.y = fma(w, y.y, rs * v[u].y);
      v[u] = y;
      prod *= w;
    }
    qlast = ep * r;
    return;
  }
  // from the closed-form pivot at the segment's first row, the recurrence
  // e_{k+1} = g + a q_k (the same operations as a single sweep)
  T e = k0 == 0 ? e0 : fma(D * z, rcp<T>((T)1 - z), ep);
  T r = rcp<T>(a + e), q = e * r;
#pragma unroll
  for (int u = 0; u < S; ++u) {
    if (u > 0) {
      e = fma(a, q, g);
      r = rcp<T>(a + e);
      q = e * r;
    }
    const bool in = FULL || u < len;
    const T ru = in ? sgn * r : (T)0;
    const T wu = in ? a * r : (T)1;
    wc[WST * u] = wu;
    y.x = fma(wu, y.x, ru * v[u].x);
    y.y = fma(wu, y.y, ru * v[u].y);
    v[u] = y;
    prod *= wu;
    if (FULL ? u == S - 1 : u == len - 1) qlast = q;
  }
}

// seg_forward for a segment whose pivots have not converged, with the pivot
// recurrence in projective form.  The excess e_k = a N_k / D_k obeys the
// linear recurrence (N, D) -> s ((1 + g/a) N + (g/a) D, N + D) (the Moebius
// map e -> g + a e / (a + e) written on homogeneous coordinates), and then
// p_k = a (N_k + D_k) / D_k, w_k = a / p_k = D_k / (N_k + D_k),
// q_k = e_k / p_k = N_k / (N_k + D_k).  Every coefficient is non-negative, so
// nothing cancels; s = 1 / (2 + g/a) bounds the dominant eigenvalue of the
// map by 1 (and from below by 1/2), so 32 rows neither overflow nor
// underflow.  The recurrence is two FMAs deep per row and the reciprocal
// is off the chain (the reciprocal recurrence has one per row on it).
// FP32 only.
template <int S, bool FULL, int WST = 32>
__device__ __forceinline__ void seg_forward_lin(cplx<float> (&v)[S], int len, int k0, float a, float g, float e0,
                                                float sgn, float ep, float D, float z, float *wc, cplx<float> &y,
                                                float &prod, float &qlast) {
  y = mk<float>(0, 0);
  prod = 1.f;
  qlast = 0.f;
  const float ia = rcp<float>(a), gh = g * ia;
  const float sc = rcp<float>(2.f + gh);
  const float c11 = sc * (1.f + gh), c12 = sc * gh;
  const float e = k0 == 0 ? e0 : fmaf(D * z, rcp<float>(1.f - z), ep);
  float Nn = e * ia, Dd = 1.f;
  const float rs = sgn * ia;
#pragma unroll
  for (int u = 0; u < S; ++u) {
    const float t = Nn + Dd;
    const float it = rcp<float>(t);
    const float w = Dd * it;
    const bool in = FULL || u < len;
    const float wu = in ? w : 1.f;
    const float ru = in ? rs * w : 0.f;
    wc[WST * u] = wu;
    y.x = fmaf(wu, y.x, ru * v[u].x);
    y.y = fmaf(wu, y.y, ru * v[u].y);
    v[u] = y;
    prod *= wu;
    if (FULL ? u == S - 1 : u == len - 1) qlast = Nn * it;
    const float nN = fmaf(c11, Nn, c12 * Dd);
    Dd = sc * t;
    Nn = nN;
  }
}

// Carry c (y before the segment) folded in, then the local back substitution
// from a zero carry; returns xhat at the segment's first row.
template <typename T, int S, bool FULL, bool CW, int WST = 32>
__device__ __forceinline__ cplx<T> seg_middle(cplx<T> (&v)[S], int len, T wconst, const T *wc, cplx<T> c) {
  T pw = (T)1;
#pragma unroll
  for (int u = 0; u < S; ++u) {
    pw *= CW ? wconst : wc[WST * u];
    const bool in = FULL || u < len;
    v[u].x = in ? fma(pw, c.x, v[u].x) : (T)0;
    v[u].y = in ? fma(pw, c.y, v[u].y) : (T)0;
  }
  cplx<T> x = mk<T>(0, 0);
#pragma unroll
  for (int u = S - 1; u >= 0; --u) {
    const T wu = CW ? wconst : wc[WST * u];
    x.x = fma(wu, x.x, v[u].x);
    x.y = fma(wu, x.y, v[u].y);
    v[u] = x;
  }
  return x;
}

// Carry c (x after the segment) folded in and the rows stored.
template <typename T, int S, bool FULL, bool CW, int WST = 32>
__device__ __forceinline__ void seg_store(cplx<T> (&v)[S], int len, T wconst, const T *wc, cplx<T> c, bool live,
                                          cplx<T> *col, long step) {
  T pw = (T)1;
#pragma unroll
  for (int u = S - 1; u >= 0; --u) {
    pw *= CW ? wconst : wc[WST * u];
    cplx<T> o;
    o.x = fma(pw, c.x, v[u].x);
    o.y = fma(pw, c.y, v[u].y);
    if (live && (FULL || u < len)) col[(long)u * step] = o;
  }
}

}  // namespace ibm
