// pencil.cu -- tridiagonal solve along y for every Fourier pencil (kx, kz).
//
// After the x/z transforms each pencil obeys (Sec. 2.3.3, Eq. 5 / Appendix B)
//     M x = f,   M = tridiag(-a, 2a + g, -a)
// with the first/last diagonal a(1 + beta) + g (Neumann beta = 0, no-slip
// cell-centred beta = 2, wall-normal faces beta = 1).  Poisson: a = 1/hy^2,
// g = kx'^2 + kz'^2 (Appendix A) and f = -b_hat; Helmholtz (I - c L):
// a = c/hy^2, g = 1 + c (kx'^2 + kz'^2) and f = r_hat.
//
// Thomas' algorithm (Sec. 2.3.3, S1.1/S2.1) is run in "excess" form: every
// pivot is written p_i = a + e_i with e_0 = g + a beta_s and
// e_i = g + a q_{i-1}, q_i = e_i / p_i, so no pivot is formed as a
// difference of nearly equal numbers.  The classic recurrence p_i =
// (2a + g) - a^2/p_{i-1} loses g against 2a in FP32 for the long-wave pencils
// (g/a ~ 1e-4 at 128 points); the excess form keeps every quantity a sum of
// non-negative terms and gives FP32 pencils ~1e-6 relative accuracy.
// Forward:  y_i = r_i f_i + (1 - q_i) y_{i-1},  r_i = 1/p_i
// Backward: x_i = y_i + (1 - q_i) x_{i+1}
//
// The Poisson (0, 0) pencil is singular (Neumann at both ends).  It is
// solved in FP64 by an extra CTA of the same grid, off the critical path of
// the other pencils: the right-hand side is made compatible by removing its
// mean (reported as the removed mean of b), the paper's pin x_0 = 0 fixes
// the constant (Sec. 2.3.3, S2.1), the bidiagonal factors of the zero-mode
// matrix reduce the elimination to two running sums (a (x_{j+1} - x_j) =
// sum_{i<=j} f_i), and the FP64 mean of x is removed (mean(phi) = 0).
#include <algorithm>

#include "internal.h"
#include "seg.cuh"
#include "tma.cuh"

namespace ibm {

template <typename T> struct PencilTile { static constexpr int TP = 16; };

// The extra CTA of a pencil grid: the FP64 zero mode (returns true if this
// CTA was that one).
__device__ __forceinline__ bool zero_mode_cta(const PencilParams &pp, double *zs, double *mean_out) {
  if (!pp.zero_mode || blockIdx.x != gridDim.x - 1) return false;
  if (threadIdx.x < 32)
    zero_mode_fp64(pp.zrhs, pp.zsol, zs, pp.ny, pp.inv_ny, pp.hy2, pp.inv_nxnz, mean_out);
  return true;
}

// Two lanes per pencil, Thomas in excess form from both ends ("twisted"
// elimination): the even lane eliminates rows 0 .. m-1 top-down, the odd
// lane rows n-1 .. m+1 bottom-up, and the two meet at row m = n/2, where
//   (g + a q^T_{m-1} + a q^B_{m+1}) x_m = f_m + a (y^T_{m-1} + y^B_{m+1})
// (a sum of non-negative terms, like every other pivot).  Each lane then
// substitutes back towards its end.  The serial depth per pencil is n
// instead of 2n.  Per row of a half sweep (r = 1/(a + e), w = a r = 1 - q):
//   forward   y_s = r f_s + w y_{s-1}      (y over f in the shared tile, w kept)
//   backward  x_s = y_s + w_s x_{s+1}      (straight to the spectrum)
template <typename T>
__device__ __forceinline__ void half_forward(cplx<T> *t, int stp, T *wc, int len, T a, T g, T e0, T sgn, cplx<T> &y,
                                             T &q) {
  T e = e0;
  y.x = (T)0;
  y.y = (T)0;
#pragma unroll 4
  for (int s = 0; s < len; ++s) {
    const cplx<T> f = t[s * stp];
    if (s > 0) e = fma(a, q, g);
    const T r = rcp<T>(a + e);
    q = e * r;
    const T w = a * r;
    y.x = fma(r, sgn * f.x, w * y.x);
    y.y = fma(r, sgn * f.y, w * y.y);
    t[s * stp] = y;
    wc[s * stp] = w;
  }
}

template <typename T>
__device__ __forceinline__ void half_backward(const cplx<T> *t, int stp, const T *wc, int len, cplx<T> x,
                                              cplx<T> *gcol, long gstep) {
#pragma unroll 4
  for (int s = len - 1; s >= 0; --s) {
    const cplx<T> y = t[s * stp];
    const T w = wc[s * stp];
    x.x = fma(w, x.x, y.x);
    x.y = fma(w, x.y, y.y);
    gcol[s * gstep] = x;
  }
}

// Variant for grids with more pencils than the tile kernel keeps resident:
// no tile; the forward half sweep writes y_s over f_s in the spectrum itself
// (loads run U to 2U rows ahead of the recurrence), only w stays in shared
// memory, and the backward sweep reads y_s back (mostly from L2).
template <typename T> struct SweepDepth { static constexpr int U = 16; };
template <> struct SweepDepth<double> { static constexpr int U = 8; };

template <typename T, int U>
__device__ __forceinline__ void gl_forward(cplx<T> *col, long step, T *wc, int wstep, int len, T a, T g, T e0, T sgn,
                                           cplx<T> &y, T &q) {
  cplx<T> fb[U];
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (u < len) fb[u] = col[u * step];
  T e = e0;
  y.x = (T)0;
  y.y = (T)0;
  for (int s0 = 0; s0 < len; s0 += U) {
    cplx<T> fn[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (s0 + U + u < len) fn[u] = col[(s0 + U + u) * step];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u;
      if (s < len) {
        if (s > 0) e = fma(a, q, g);
        const T r = rcp<T>(a + e);
        q = e * r;
        const T w = a * r;
        y.x = fma(r, sgn * fb[u].x, w * y.x);
        y.y = fma(r, sgn * fb[u].y, w * y.y);
        col[s * step] = y;
        wc[s * wstep] = w;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) fb[u] = fn[u];
  }
}

template <typename T, int U>
__device__ __forceinline__ void gl_backward(cplx<T> *col, long step, const T *wc, int wstep, int len, cplx<T> x) {
  cplx<T> yb[U];
  T wb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int s = len - 1 - u;
    if (s >= 0) { yb[u] = col[s * step]; wb[u] = wc[s * wstep]; }
  }
  for (int s0 = len - 1; s0 >= 0; s0 -= U) {
    cplx<T> yn[U];
    T wn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 - U - u;
      if (s >= 0) { yn[u] = col[s * step]; wn[u] = wc[s * wstep]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 - u;
      if (s >= 0) {
        x.x = fma(wb[u], x.x, yb[u].x);
        x.y = fma(wb[u], x.y, yb[u].y);
        col[s * step] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) { yb[u] = yn[u]; wb[u] = wn[u]; }
  }
}

template <typename T>
__global__ void __launch_bounds__(32)
k_pencil_g(Ptr3<cplx<T> *> S_, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
           double *mean_out) {
  pdl_wait();
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  int beta_s, beta_e, j0;
  pencil_field(pp, blockIdx.y, beta_s, beta_e, j0);
  constexpr int TP = PencilTile<T>::TP;
  constexpr int U = SweepDepth<T>::U;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = pp.ny - j0;
  T *ws = reinterpret_cast<T *>(smem_raw);                     // [n][TP]
  double *zs = reinterpret_cast<double *>(ws + (size_t)pp.ny * TP);  // [ny] (zero-mode CTA)
  if (zero_mode_cta(pp, zs, mean_out)) return;
  const long plane = (long)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int lane = threadIdx.x;
  const int bottom = lane & 1, pl = lane >> 1;
  const int p = blockIdx.x * TP + pl;
  const bool live = p < npen && !(pp.zero_mode && p == 0);
  const int m = n / 2;
  const int len = bottom ? n - 1 - m : m;
  const int pc = live ? p : 0;
  const int kz = pc / pp.P, kx = pc - kz * pp.P;
  const T a = (T)pp.a;
  const T g = (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]);
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  cplx<T> *c0 = S + pc + (long)j0 * plane;  // row 0 of the unknowns
  const int first = bottom ? n - 1 : 0;
  cplx<T> *col = c0 + (long)first * plane;
  const long step = bottom ? -plane : plane;
  T *wc = ws + first * TP + pl;
  const int wstep = bottom ? -TP : TP;
  const T e0 = g + a * (T)(bottom ? beta_e : beta_s);
  cplx<T> y;
  T q = (T)0;
  if (live) gl_forward<T, U>(col, step, wc, wstep, len, a, g, e0, sgn, y, q);
  // meet at row m: the top lane reads f_m, the pair swaps (y, q) and f_m
  cplx<T> f;
  f.x = (T)0;
  f.y = (T)0;
  if (live && !bottom) f = c0[(long)m * plane];
  const T yo_x = __shfl_xor_sync(0xffffffffu, y.x, 1);
  const T yo_y = __shfl_xor_sync(0xffffffffu, y.y, 1);
  const T qo = __shfl_xor_sync(0xffffffffu, q, 1);
  const T fo_x = __shfl_xor_sync(0xffffffffu, f.x, 1);
  const T fo_y = __shfl_xor_sync(0xffffffffu, f.y, 1);
  if (!live) return;
  if (bottom) { f.x = fo_x; f.y = fo_y; }
  cplx<T> x;
  {
    const T rm = rcp<T>(g + a * q + a * qo);
    x.x = (sgn * f.x + a * (y.x + yo_x)) * rm;
    x.y = (sgn * f.y + a * (y.y + yo_y)) * rm;
  }
  if (!bottom) c0[(long)m * plane] = x;
  gl_backward<T, U>(col, step, wc, wstep, len, x);
  if (j0 == 1 && !bottom) {
    cplx<T> z; z.x = (T)0; z.y = (T)0;
    S[p] = z;
  }
}

template <typename T>
__global__ void __launch_bounds__(32)
k_pencil(Ptr3<cplx<T> *> S_, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
         double *mean_out) {
  pdl_wait();
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  int beta_s, beta_e, j0;
  pencil_field(pp, blockIdx.y, beta_s, beta_e, j0);
  constexpr int TP = PencilTile<T>::TP;  // pencils per CTA, two lanes each
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ny = pp.ny;
  const int n = ny - j0;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw + 16);  // [n][TP], rows 16-byte aligned for the bulk copies
  T *ws = reinterpret_cast<T *>(tile + (size_t)n * TP);        // [n][TP]
  double *zs = reinterpret_cast<double *>(ws + (size_t)n * TP);  // [ny] (zero-mode CTA, n = ny)
  if (zero_mode_cta(pp, zs, mean_out)) return;
  const long plane = (long)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int p0 = blockIdx.x * TP;
  const int np = min(TP, npen - p0);  // even: npen is even and p0 a multiple of TP
  const int lane = threadIdx.x;
  const cplx<T> *src = S + (long)j0 * plane + p0;
  // rows of the tile arrive by bulk copy (np * 8 or 16 bytes each)
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(cplx<T>) * np * n));
  }
  __syncwarp();
  for (int j = lane; j < n; j += 32)
    bulk_g2s(tile + (size_t)j * TP, src + (long)j * plane, (uint32_t)(sizeof(cplx<T>) * np), bar);
  if (!__all_sync(0xffffffffu, mbar_wait(bar, 0, pp.err))) {
    mbar_wait(bar, 0, nullptr);  // copies still in flight must land before the CTA's memory is reused
    return;
  }
  const int bottom = lane & 1, pl = lane >> 1;
  const int p = p0 + pl;
  // the (0,0) pencil is singular (g = 0): its sweep is skipped here and its
  // FP64 solution reaches the inverse transform through zsol
  const bool live = pl < np && !(pp.zero_mode && p == 0);
  const int m = n / 2;
  const int len = bottom ? n - 1 - m : m;
  const int pc = live ? p : 0;
  const int kz = pc / pp.P, kx = pc - kz * pp.P;
  const T a = (T)pp.a;
  const T g = (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]);
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const int first = bottom ? n - 1 : 0;
  const int stp = bottom ? -TP : TP;
  cplx<T> *t = tile + first * TP + pl;
  T *wc = ws + first * TP + pl;
  const T e0 = g + a * (T)(bottom ? beta_e : beta_s);
  cplx<T> y;
  T q = (T)0;
  if (live) half_forward<T>(t, stp, wc, len, a, g, e0, sgn, y, q);
  // meet at row m
  const T yo_x = __shfl_xor_sync(0xffffffffu, y.x, 1);
  const T yo_y = __shfl_xor_sync(0xffffffffu, y.y, 1);
  const T qo = __shfl_xor_sync(0xffffffffu, q, 1);
  if (!live) return;
  cplx<T> *gcol = S + p + (long)j0 * plane;  // row 0 of the unknowns in the spectrum
  cplx<T> x;
  {
    const cplx<T> f = tile[m * TP + pl];
    const T rm = rcp<T>(g + a * q + a * qo);
    x.x = (sgn * f.x + a * (y.x + yo_x)) * rm;
    x.y = (sgn * f.y + a * (y.y + yo_y)) * rm;
  }
  if (!bottom) gcol[(long)m * plane] = x;
  half_backward<T>(t, stp, wc, len, x, gcol + (long)first * plane, bottom ? -plane : plane);
  if (j0 == 1 && !bottom) {
    cplx<T> z; z.x = (T)0; z.y = (T)0;
    S[p] = z;
  }
}

// ---------------------------------------------------------------------------
// Segmented two-ended sweep: one CTA takes 32 consecutive pencils (lane =
// pencil, so every row access is a run of 32 complex values) and L = 2 Lh
// warps.  The elimination order is the two-ended one of k_pencil (rows
// 0 .. m-1 top-down, rows n-1 .. m+1 bottom-up, meeting at m = n/2); warps
// 0 .. Lh-1 share the top half and Lh .. L-1 the bottom half, S rows each,
// held in registers.  Along each half, with k the distance from the wall:
//   * pivots: e_k depends on the pencil's (a, g) only.  The map
//     e -> g + a e / (a + e) is a Moebius map with fixed points e+ > 0 and
//     e- = -a g / e+, and z_k = (e_k - e+) / (e_k - e-) shrinks
//     geometrically, z_k = z_0 lambda^k with 1 - lambda =
//     (a g + e+^2) / (e+ (a + e+)), so the pivot at any row follows in closed
//     form, e_k = e+ + (e+ - e-) z_k / (1 - z_k) (all terms sums and
//     products of positive numbers but z, whose absolute error only moves
//     e_k by a few ulps of e+, far below the pivot a + e_k).  A warp takes
//     its first row's pivot from it and runs the recurrence through its own
//     rows, or, when all its lanes have |z| below a sixteenth of the unit
//     roundoff there, the converged pivot e+ for every row (constant r, w);
//   * forward elimination y_k = r_k f_k + w_k y_{k-1} (w = a r) is a
//     first-order linear recurrence: each warp sweeps its rows from a zero
//     carry, keeping yhat and the product of its w, and the true values
//     follow from the warps' (yhat_end, prod w) pairs in shared memory,
//     y_k = yhat_k + (w_s ... w_k) y_{s-1};
//   * every thread then forms x_m from both halves' last y and q, and back
//     substitution x_k = y_k + w_k x_{k+1} runs the same way towards the wall.
// One global read and one write of the spectrum; the serial depth per warp
// is S rows of the y and x recurrences.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cp_async_elem(cplx<T> *dst, const cplx<T> *src) {
  if constexpr (sizeof(T) == 4) cp_async8(dst, src);
  else cp_async16(dst, src);
}

template <typename T, int S, int MAXT> struct SegOcc {
  // resident CTAs per SM the register budget is sized for (shared memory
  // allows about as many)
  static constexpr int value = MAXT > 256 ? 1 : (S >= 32 || sizeof(T) == 8 ? 2 : (S >= 16 ? 3 : 4));
};

// Per-lane constants of one tile (32 pencils of one field).
template <typename T> struct SegTile {
  cplx<T> *Sb, *c0, *col;
  long step;
  T g, e0;
  int n, m, k0, len, beta_s, beta_e, j0, p;
  bool live;
};

template <typename T, int S>
__device__ __forceinline__ SegTile<T> seg_tile(const PencilParams &pp, Ptr3<cplx<T> *> S_, const T *lamx,
                                               const T *lamz, int t, int nblk, int seg, int lane, int Lh) {
  SegTile<T> ti;
  const int field = t / nblk, blk = t - field * nblk;
  pencil_field(pp, field, ti.beta_s, ti.beta_e, ti.j0);
  ti.n = pp.ny - ti.j0;
  ti.m = ti.n / 2;
  const long plane = (long)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  ti.p = blk * 32 + lane;
  ti.live = ti.p < npen && !(pp.zero_mode && ti.p == 0);
  const int pc = ti.p < npen ? ti.p : npen - 1;  // dead lanes compute on a valid pencil, store nothing
  const int kz = pc / pp.P, kx = pc - kz * pp.P;
  ti.g = (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]);
  const bool top = seg < Lh;
  ti.e0 = ti.g + (T)pp.a * (T)(top ? ti.beta_s : ti.beta_e);
  ti.k0 = (top ? seg : seg - Lh) * S;  // distance of my first row from the wall
  const int hl = top ? ti.m : ti.n - 1 - ti.m;
  ti.len = max(0, min(S, hl - ti.k0));  // my rows (the same for every lane)
  ti.step = top ? plane : -plane;
  ti.Sb = S_[field];
  ti.c0 = ti.Sb + (long)ti.j0 * plane + pc;  // row 0 of the unknowns
  ti.col = ti.c0 + (long)(top ? ti.k0 : ti.n - 1 - ti.k0) * plane;
  return ti;
}

// The tile's rows (and, for warp 0, row m) by per-thread asynchronous copies.
template <typename T, int S>
__device__ __forceinline__ void seg_issue(const SegTile<T> &ti, cplx<T> *tl, cplx<T> *tm, int seg, long plane) {
#pragma unroll
  for (int u = 0; u < S; ++u)
    if (u < ti.len) cp_async_elem<T>(tl + 32 * u, ti.col + (long)u * ti.step);
  if (seg == 0) cp_async_elem<T>(tm, ti.c0 + (long)ti.m * plane);
}

// Persistent: CTA b takes tiles b, b + G, ... of the (field, 32-pencil block)
// list (G = the sweep CTAs); the copies of its next tile stream into the one
// staging buffer while the current tile, already in registers, is solved.
template <typename T, int S, int MAXT>
__global__ void __launch_bounds__(MAXT, (SegOcc<T, S, MAXT>::value))
k_pencil_seg(Ptr3<cplx<T> *> S_, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
             double *mean_out) {
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5, L = blockDim.x >> 5, Lh = L >> 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw);  // [L S + 1][32] rows by sweep slot, then row m
  T *ws = reinterpret_cast<T *>(tile + (size_t)(L * S + 1) * 32);  // [L S][32] w of every row
  T *cf = ws + (size_t)L * S * 32;  // [4][L][32] (yhat_end.x, .y, prod w, q of the last row)
  T *cb = cf + 4 * L * 32;          // [2][L][32] (xhat_first.x, .y)
  const int G = gridDim.x - (pp.zero_mode ? 1 : 0);
  if (pp.zero_mode && blockIdx.x == G) {
    pdl_wait();
    zero_mode_cta(pp, reinterpret_cast<double *>(cb + 2 * L * 32), mean_out);
    return;
  }
  const long plane = (long)pp.nz * pp.P;
  const int nblk = ceil_div(pp.nz * pp.P, 32);
  const int tiles = nblk * pp.nb;
  const T a = (T)pp.a;
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const bool top = seg < Lh;
  cplx<T> *tl = tile + (size_t)seg * S * 32 + lane;
  cplx<T> *tm = tile + (size_t)L * S * 32 + lane;
  T *wc = ws + (size_t)seg * S * 32 + lane;  // w of my row u at wc[32 u]
  pdl_wait();
  int t = blockIdx.x;
  if (t < tiles) seg_issue<T, S>(seg_tile<T, S>(pp, S_, lamx, lamz, t, nblk, seg, lane, Lh), tl, tm, seg, plane);
  for (; t < tiles; t += G) {
    const SegTile<T> cur = seg_tile<T, S>(pp, S_, lamx, lamz, t, nblk, seg, lane, Lh);
    const SegTile<T> &ti = cur;
    const T g = ti.g;
    const int k0 = ti.k0, len = ti.len, n = ti.n, m = ti.m;
    // pivots in closed form (fixed points e+ > 0 > e- = -a g / e+ of the
    // Moebius map, z_k = z_0 lambda^k); the singular zero pencil (g = 0)
    // keeps e = e0 = 0
    T ep, D, z;
    const bool cw = __all_sync(0xffffffffu, seg_pivots<T>(a, g, ti.e0, k0, ep, D, z)) && len == S;
    cp_async_wait_all();
    __syncthreads();  // every copy of the tile has landed
    cplx<T> v[S];
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = u < len ? tl[32 * u] : mk<T>(0, 0);
    const cplx<T> fm = *tm;
    __syncthreads();  // the staging buffer is free: start the next tile's copies
    if (t + G < tiles)
      seg_issue<T, S>(seg_tile<T, S>(pp, S_, lamx, lamz, t + G, nblk, seg, lane, Lh), tl, tm, seg, plane);
    const T wconst = a * rcp<T>(a + ep);
    cplx<T> y;
    T prod, qlast;
    if (cw) seg_forward<T, S, true, true>(v, len, k0, a, g, ti.e0, sgn, ep, D, z, wc, y, prod, qlast);
    else if constexpr (sizeof(T) == 4)  // FP32: the projective pivot recurrence (reciprocal off the chain)
      seg_forward_lin<S, false>(v, len, k0, a, g, ti.e0, sgn, ep, D, z, wc, y, prod, qlast);
    else seg_forward<T, S, false, false>(v, len, k0, a, g, ti.e0, sgn, ep, D, z, wc, y, prod, qlast);
    cf[(0 * L + seg) * 32 + lane] = y.x;
    cf[(1 * L + seg) * 32 + lane] = y.y;
    cf[(2 * L + seg) * 32 + lane] = prod;
    cf[(3 * L + seg) * 32 + lane] = qlast;
    __syncthreads();
    // y at the row before mine, and the last y of both halves
    cplx<T> c = mk<T>(0, 0);
    cplx<T> yT = mk<T>(0, 0), yB = mk<T>(0, 0);
    for (int s2 = 0; s2 < L; ++s2) {
      if (s2 == seg) c = s2 < Lh ? yT : yB;
      const T pw = cf[(2 * L + s2) * 32 + lane];
      const T ax = cf[(0 * L + s2) * 32 + lane], ay = cf[(1 * L + s2) * 32 + lane];
      if (s2 < Lh) {
        yT.x = fma(pw, yT.x, ax);
        yT.y = fma(pw, yT.y, ay);
      } else {
        yB.x = fma(pw, yB.x, ax);
        yB.y = fma(pw, yB.y, ay);
      }
    }
    // meeting row: (g + a q^T + a q^B) x_m = f_m + a (y^T_{m-1} + y^B_{m+1});
    // an empty half contributes its wall term beta
    const T qT = m > 0 ? cf[(3 * L + (m - 1) / S) * 32 + lane] : (T)cur.beta_s;
    const T qB = n - 1 - m > 0 ? cf[(3 * L + Lh + (n - 2 - m) / S) * 32 + lane] : (T)cur.beta_e;
    cplx<T> xm;
    {
      const T rm = rcp<T>(g + a * qT + a * qB);
      xm.x = (sgn * fm.x + a * (yT.x + yB.x)) * rm;
      xm.y = (sgn * fm.y + a * (yT.y + yB.y)) * rm;
    }
    cplx<T> x;
    if (cw) x = seg_middle<T, S, true, true>(v, len, wconst, wc, c);
    else x = seg_middle<T, S, false, false>(v, len, wconst, wc, c);
    cb[(0 * L + seg) * 32 + lane] = x.x;
    cb[(1 * L + seg) * 32 + lane] = x.y;
    __syncthreads();
    c = xm;  // x at the row after my last one (towards the meeting row)
    for (int s2 = (top ? Lh : L) - 1; s2 > seg; --s2) {
      const T pw = cf[(2 * L + s2) * 32 + lane];
      c.x = fma(pw, c.x, cb[(0 * L + s2) * 32 + lane]);
      c.y = fma(pw, c.y, cb[(1 * L + s2) * 32 + lane]);
    }
    if (cw) seg_store<T, S, true, true>(v, len, wconst, wc, c, cur.live, cur.col, cur.step);
    else seg_store<T, S, false, false>(v, len, wconst, wc, c, cur.live, cur.col, cur.step);
    if (seg == 0 && cur.live) {
      cur.c0[(long)m * plane] = xm;
      if (cur.j0 == 1) cur.Sb[cur.p] = mk<T>(0, 0);
    }
  }
}

template <typename T, int S> size_t pencil_seg_smem_bytes(int L, int ny) {
  const size_t body = sizeof(cplx<T>) * (size_t)(L * S + 1) * 32 + sizeof(T) * ((size_t)L * S + 6 * L) * 32;
  return ((body + 15) & ~(size_t)15) + (size_t)ny * sizeof(double);
}

template <typename T, int S, int MAXT>
static cudaError_t launch_seg(const PencilParams &pp, Ptr3<cplx<T> *> S3, const T *lamx, const T *lamz,
                              double *mean_out, cudaStream_t st) {
  const int L = 2 * ceil_div(pp.ny / 2, S);  // both halves of every field (n = ny or ny - 1 rows)
  if (32 * L > MAXT) return cudaErrorInvalidConfiguration;
  {
    cudaError_t e = ensure_max_smem<k_pencil_seg<T, S, MAXT>>();
    if (e != cudaSuccess) return e;
  }
  const size_t bytes = pencil_seg_smem_bytes<T, S>(L, pp.ny);
  static std::once_flag once;
  static int sms = 0;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  int per_sm = 0;
  IBM_KTRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pencil_seg<T, S, MAXT>, 32 * L, bytes));
  const int tiles = ceil_div(pp.nz * pp.P, 32) * pp.nb;
  const int G = std::max(1, std::min(tiles, sms * std::max(per_sm, 1)));
  IBM_KTRY(launch_pdl(k_pencil_seg<T, S, MAXT>, G + (pp.zero_mode ? 1 : 0), 32 * L, bytes, st, S3, lamx, lamz, pp,
                      mean_out));
  return cudaGetLastError();
}

// Rows per warp of the segmented sweep for ny rows (0: not available; the
// CTA has 2 ceil((ny / 2) / S) warps).
template <typename T> static int seg_rows(int ny) {
  if (ny < 4) return 0;
  if (ny <= 64) return 8;
  if (ny <= 128) return 16;
  if (ny <= 256) return sizeof(T) == 4 ? 32 : 16;
  return (sizeof(T) == 4 && ny <= 512) ? 32 : 0;
}

// ---------------------------------------------------------------------------
// Substructured pencil solve: one CTA of 32 warps takes TP pencils; warp s
// owns the block of rows [s M, (s+1) M) of every pencil, lane = pencil (or,
// with SPLIT, lane = (pencil, real component) for 16 pencils).  Per block:
//   * the last row of every block except the last is a separator; the other
//     rows are interior and form the local matrix M_s (excess-form LU);
//   * local solves give, at the block ends, v = M_s^-1 (a e_first),
//     w = M_s^-1 (a e_last), z = M_s^-1 ex (ex = row excess of the pencil
//     matrix, so v + w + z = 1 and the separator excess
//     ex_r + a z_last + a z_first(next) is a sum of positive terms) and
//     y = M_s^-1 f;
//   * the separator rows form a tridiagonal M-matrix solved by parallel
//     cyclic reduction over the 32 warps in excess form (row excess
//     E' = E + alpha E_up + gamma E_down);
//   * each block re-solves its interior with the separators folded into
//     the right-hand side.
// The serial depth per pencil drops from 2 ny to about 4 M + 5 levels.
// ---------------------------------------------------------------------------
template <typename T, int M, bool SPLIT> struct SsCfg {
  static constexpr int NW = 32;
  static constexpr int TP = SPLIT ? 16 : 32;
  static constexpr int NC = SPLIT ? 1 : 2;
};

// 1 when i == target else 0, as the working type (masks instead of runtime indexing)
template <typename T> __device__ __forceinline__ T pick_t(int i, int target) { return i == target ? (T)1 : (T)0; }

template <typename T, int M>
__device__ __forceinline__ void local_lu(int nint, int r0, bool has_sep, int n, T a, T g, T abs_, T abe,
                                         T (&q)[M], T (&rr)[M]) {
  T qp = (T)0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (i < nint) {
      const int row = r0 + i;
      T exl = g + (row == 0 ? abs_ : (T)0) + (row == n - 1 ? abe : (T)0);
      if (i == 0 && r0 > 0) exl += a;
      if (i == nint - 1 && has_sep) exl += a;
      const T E = exl + (i > 0 ? a * qp : (T)0);
      const T piv = E + (i < nint - 1 ? a : (T)0);
      rr[i] = rcp<T>(piv);
      q[i] = E * rr[i];
      qp = q[i];
    }
  }
}

// In-place local solve of M_s x = rhs (rows i < nint).
template <typename T, int M>
__device__ __forceinline__ void local_solve(int nint, T a, const T (&q)[M], const T (&rr)[M], T (&x)[M]) {
  T yp = (T)0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (i < nint) {
      T y;
      if (i == 0) y = x[i] * rr[i];
      else if (i < nint - 1) y = fma(rr[i], x[i], fma(-q[i], yp, yp));
      else y = (x[i] + a * yp) * rr[i];
      x[i] = y;
      yp = y;
    }
  }
  T xn = (T)0;
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    if (i < nint) {
      if (i < nint - 1) x[i] = fma(-q[i], xn, xn) + x[i];
      xn = x[i];
    }
  }
}

template <typename T, int M, bool SPLIT>
__global__ void __launch_bounds__(1024)
k_pencil_ss(cplx<T> *__restrict__ S, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
            double *mean_out) {
  pdl_wait();
  using C = SsCfg<T, M, SPLIT>;
  constexpr int NW = C::NW, TP = C::TP, NC = C::NC;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ny = pp.ny;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw + 16);            // [ny][TP]
  T *fst = reinterpret_cast<T *>(tile + (size_t)ny * TP);               // [2+NC][NW][32] w_first, z_first, y_first
  T *sep = fst + (2 + NC) * NW * 32;                                    // [3+NC][NW][32] L, U, E, F
  double *zs = reinterpret_cast<double *>(sep + (3 + NC) * NW * 32);    // [ny]
  if (zero_mode_cta(pp, zs, mean_out)) return;
  const size_t plane = (size_t)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int p0 = blockIdx.x * TP;
  const int np = min(TP, npen - p0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(cplx<T>) * np * ny));
  }
  __syncthreads();
  if (warp == 0)
    for (int j = lane; j < ny; j += 32)
      bulk_g2s(tile + (size_t)j * TP, S + (size_t)j * plane + p0, (uint32_t)(sizeof(cplx<T>) * np), bar);
  if (!__syncthreads_and(mbar_wait(bar, 0, pp.err))) {
    mbar_wait(bar, 0, nullptr);  // copies still in flight must land before the CTA's memory is reused
    return;
  }


  const int c = SPLIT ? (lane >> 1) : lane;
  const int comp = SPLIT ? (lane & 1) : 0;
  const bool valid = c < np;
  const int p = p0 + (valid ? c : 0);
  const int kz = p / pp.P, kx = p - kz * pp.P;
  const T a = (T)pp.a;
  const T g = valid ? (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]) : (T)1;
  const T abs_ = a * (T)pp.beta_s, abe = a * (T)pp.beta_e;
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const int j0 = pp.j0;
  const int n = ny - j0;
  const int s_last = (n - 1) / M;
  const int s = warp;
  const int r0 = s * M;
  const int cnt = max(0, min(M, n - r0));
  const bool has_sep = cnt > 0 && s < s_last;
  const int nint = has_sep ? cnt - 1 : cnt;

  auto pick = [](int i, int target) { return pick_t<T>(i, target); };
  // right-hand side of this block (interior rows then the separator)
  T f[NC][M];
  T fsep[NC];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (i < cnt) {
      const cplx<T> v = tile[(size_t)(j0 + r0 + i) * TP + c];
      if (SPLIT) {
        f[0][i] = sgn * (comp ? v.y : v.x);
      } else {
        f[0][i] = sgn * v.x;
        f[NC - 1][i] = sgn * v.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < NC; ++k) f[k][i] = (T)0;
    }
  }
  // element cnt-1 picked by an arithmetic mask (a runtime index would move f to local memory)
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    fsep[k] = (T)0;
#pragma unroll
    for (int i = 0; i < M; ++i) fsep[k] = fma(pick(i, has_sep ? cnt - 1 : -1), f[k][i], fsep[k]);
  }

  T q[M], rr[M], x[M];
  local_lu<T, M>(nint, r0, has_sep, n, a, g, abs_, abe, q, rr);
  T v_last = 0, w_first = 0, z_first = 0, z_last = 0, y_first[NC], y_last[NC];
  if (nint > 0) {
    // v = M_s^-1 (a e_first) when a left separator exists
#pragma unroll
    for (int i = 0; i < M; ++i) x[i] = (i == 0 && r0 > 0) ? a : (T)0;
    local_solve<T, M>(nint, a, q, rr, x);
#pragma unroll
    for (int i = 0; i < M; ++i) v_last = fma(pick(i, nint - 1), x[i], v_last);
    // w = M_s^-1 (a e_last) when this block ends in a separator
#pragma unroll
    for (int i = 0; i < M; ++i) x[i] = (i == nint - 1 && has_sep) ? a : (T)0;
    local_solve<T, M>(nint, a, q, rr, x);
    w_first = x[0];
    // z = M_s^-1 ex
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int row = r0 + i;
      x[i] = g + (row == 0 ? abs_ : (T)0) + (row == n - 1 ? abe : (T)0);
    }
    local_solve<T, M>(nint, a, q, rr, x);
    z_first = x[0];
#pragma unroll
    for (int i = 0; i < M; ++i) z_last = fma(pick(i, nint - 1), x[i], z_last);
    // y = M_s^-1 f
#pragma unroll
    for (int k = 0; k < NC; ++k) {
#pragma unroll
      for (int i = 0; i < M; ++i) x[i] = f[k][i];
      local_solve<T, M>(nint, a, q, rr, x);
      y_first[k] = x[0];
      y_last[k] = (T)0;
#pragma unroll
      for (int i = 0; i < M; ++i) y_last[k] = fma(pick(i, nint - 1), x[i], y_last[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) { y_first[k] = (T)0; y_last[k] = (T)0; }
  }
  // publish the first-row values for the separator above
  fst[(0 * NW + s) * 32 + lane] = w_first;
  fst[(1 * NW + s) * 32 + lane] = z_first;
#pragma unroll
  for (int k = 0; k < NC; ++k) fst[((2 + k) * NW + s) * 32 + lane] = y_first[k];
  __syncthreads();
  // separator row of this block (dummy identity rows elsewhere)
  T L = 0, U = 0, E = 1, F[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) F[k] = (T)0;
  if (has_sep) {
    const int rs = r0 + cnt - 1;
    E = g + (rs == 0 ? abs_ : (T)0);
#pragma unroll
    for (int k = 0; k < NC; ++k) F[k] = fsep[k];
    if (nint > 0) {
      L = a * v_last;
      E += a * z_last;
#pragma unroll
      for (int k = 0; k < NC; ++k) F[k] += a * y_last[k];
    } else if (rs > 0) {
      L = a;
    }
    const int sn = s + 1;
    const int cntn = max(0, min(M, n - sn * M));
    const bool hsn = cntn > 0 && sn < s_last;
    const int nintn = hsn ? cntn - 1 : cntn;
    if (nintn > 0) {
      U = a * fst[(0 * NW + sn) * 32 + lane];
      E += a * fst[(1 * NW + sn) * 32 + lane];
#pragma unroll
      for (int k = 0; k < NC; ++k) F[k] += a * fst[((2 + k) * NW + sn) * 32 + lane];
    } else {
      U = a;
    }
  }
  // parallel cyclic reduction over the NW separator rows (excess form)
#define IBM_SEP(q_, row) sep[((q_) * NW + (row)) * 32 + lane]
  IBM_SEP(0, s) = L; IBM_SEP(1, s) = U; IBM_SEP(2, s) = E;
#pragma unroll
  for (int k = 0; k < NC; ++k) IBM_SEP(3 + k, s) = F[k];
  __syncthreads();
#pragma unroll
  for (int st = 1; st < NW; st <<= 1) {
    T nL = 0, nU = 0, nE = E, nF[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) nF[k] = F[k];
    if (s - st >= 0) {
      const T Lu = IBM_SEP(0, s - st), Uu = IBM_SEP(1, s - st), Eu = IBM_SEP(2, s - st);
      const T al = L * rcp<T>(Lu + Uu + Eu);
      nL = al * Lu;
      nE += al * Eu;
#pragma unroll
      for (int k = 0; k < NC; ++k) nF[k] += al * IBM_SEP(3 + k, s - st);
    }
    if (s + st < NW) {
      const T Ld = IBM_SEP(0, s + st), Ud = IBM_SEP(1, s + st), Ed = IBM_SEP(2, s + st);
      const T ga = U * rcp<T>(Ld + Ud + Ed);
      nU = ga * Ud;
      nE += ga * Ed;
#pragma unroll
      for (int k = 0; k < NC; ++k) nF[k] += ga * IBM_SEP(3 + k, s + st);
    }
    __syncthreads();
    L = nL; U = nU; E = nE;
#pragma unroll
    for (int k = 0; k < NC; ++k) F[k] = nF[k];
    IBM_SEP(0, s) = L; IBM_SEP(1, s) = U; IBM_SEP(2, s) = E;
#pragma unroll
    for (int k = 0; k < NC; ++k) IBM_SEP(3 + k, s) = F[k];
    __syncthreads();
  }
  // separator values X_s = F / E (all couplings eliminated); publish
  const T rE = rcp<T>(E);
#pragma unroll
  for (int k = 0; k < NC; ++k) IBM_SEP(3 + k, s) = F[k] * rE;
  __syncthreads();
  if (cnt > 0) {
    T XL[NC], XR[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      XL[k] = s > 0 ? IBM_SEP(3 + k, s - 1) : (T)0;
      XR[k] = has_sep ? IBM_SEP(3 + k, s) : (T)0;
    }
    // re-solve the interior with the separators folded in
    T out[NC][M];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        T r = f[k][i];
        if (i == 0 && r0 > 0) r += a * XL[k];
        if (i == nint - 1 && has_sep) r += a * XR[k];
        x[i] = r;
      }
      if (nint > 0) local_solve<T, M>(nint, a, q, rr, x);
#pragma unroll
      for (int i = 0; i < M; ++i) out[k][i] = (i < nint) ? x[i] : XR[k];
    }
    if (valid) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        if (i < cnt) {
          cplx<T> *dst = tile + (size_t)(j0 + r0 + i) * TP + c;
          if (SPLIT) {
            if (comp) dst->y = out[0][i];
            else dst->x = out[0][i];
          } else {
            dst->x = out[0][i];
            dst->y = out[NC - 1][i];
          }
        }
      }
    }
  }
#undef IBM_SEP
  if (j0 == 1 && warp == 0 && lane < TP) {
    cplx<T> z; z.x = (T)0; z.y = (T)0;
    tile[lane] = z;
  }
  fence_proxy_async();
  __syncthreads();
  if (warp == 0) {
    for (int j = lane; j < ny; j += 32)
      bulk_s2g(S + (size_t)j * plane + p0, tile + (size_t)j * TP, (uint32_t)(sizeof(cplx<T>) * np));
    bulk_commit();
    bulk_wait_read();
  }
}

template <typename T, int M, bool SPLIT> size_t pencil_ss_smem_bytes(int ny) {
  using C = SsCfg<T, M, SPLIT>;
  return 16 + (size_t)ny * C::TP * sizeof(cplx<T>) + sizeof(T) * (size_t)((2 + C::NC) + (3 + C::NC)) * C::NW * 32 +
         (size_t)ny * sizeof(double);
}

template <typename T, int M, bool SPLIT>
static cudaError_t launch_ss(const PencilParams &pp, cplx<T> *S, const T *lamx, const T *lamz, double *mean_out,
                             cudaStream_t st) {
  using C = SsCfg<T, M, SPLIT>;
  const size_t bytes = pencil_ss_smem_bytes<T, M, SPLIT>(pp.ny);
  {
    cudaError_t e = ensure_max_smem<k_pencil_ss<T, M, SPLIT>>();
    if (e != cudaSuccess) return e;
  }
  const int npen = pp.nz * pp.P;
  IBM_KTRY(launch_pdl(k_pencil_ss<T, M, SPLIT>, ceil_div(npen, C::TP) + (pp.zero_mode ? 1 : 0), 1024, bytes, st, S, lamx, lamz, pp,
                                                                                             mean_out));
  return cudaGetLastError();
}

template <typename T> size_t pencil_smem_bytes(int ny) {
  constexpr int TP = PencilTile<T>::TP;
  return 16 + (size_t)ny * sizeof(double) + (size_t)ny * TP * (sizeof(cplx<T>) + sizeof(T));
}
template <typename T> size_t pencil_g_smem_bytes(int ny) {
  constexpr int TP = PencilTile<T>::TP;
  return (size_t)ny * sizeof(double) + (size_t)ny * TP * sizeof(T);
}

// Resident 32-thread CTAs of a kernel with `bytes` of dynamic shared memory
// on the whole device (per-device attributes read once).
static long resident_ctas(size_t bytes) {
  static std::once_flag once;
  static int sms = 0, smem = 0;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  });
  const long per_sm = std::min<long>(32, (long)smem / (long)(bytes + 1024));
  return (long)sms * std::max<long>(per_sm, 1);
}

template <typename T>
cudaError_t launch_pencil(const PencilParams &pp, Ptr3<cplx<T> *> S3, const T *lamx, const T *lamz, double *mean_out,
                          cudaStream_t st) {
  if (pp.periodic)
    return launch_ypencil<T>(pp, S3, static_cast<const cplx<T> *>(pp.twy), lamx, lamz,
                             static_cast<const T *>(pp.lamy), mean_out, st);
  if (pp.mode == 1 && pp.nb > 1) {
    // the warp-parallel block solve takes one field per launch
    for (int b = 0; b < pp.nb; ++b) {
      PencilParams q = pp;
      q.nb = 1;
      if (b > 0) { q.beta_s = pp.fbc[b] & 15; q.beta_e = (pp.fbc[b] >> 4) & 15; q.j0 = pp.fbc[b] >> 8; }
      cudaError_t e = launch_pencil<T>(q, ptr3<cplx<T> *>(S3[b]), lamx, lamz, mean_out, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // default: the segmented sweep for FP32 (measured faster at 128^3 and
  // 256^3); FP64 is bound by its divisions and stays on the two-ended sweep
  if (pp.mode == 4 || (pp.mode == 0 && sizeof(T) == 4 && seg_rows<T>(pp.ny) > 0)) {
    switch (seg_rows<T>(pp.ny)) {
      case 8: return launch_seg<T, 8, 256>(pp, S3, lamx, lamz, mean_out, st);
      case 16: return launch_seg<T, 16, sizeof(T) == 4 ? 256 : 512>(pp, S3, lamx, lamz, mean_out, st);
      case 32:
        if constexpr (sizeof(T) == 4) {
          if (pp.ny <= 256) return launch_seg<T, 32, 256>(pp, S3, lamx, lamz, mean_out, st);
          return launch_seg<T, 32, 512>(pp, S3, lamx, lamz, mean_out, st);
        }
        break;
      default: break;
    }
  }
  cplx<T> *S = S3[0];
  const int n = pp.ny - pp.j0;
  if (pp.mode == 1) {
    if constexpr (sizeof(T) == 4) {
      if (n <= 32) return launch_ss<T, 1, false>(pp, S, lamx, lamz, mean_out, st);
      if (n <= 64) return launch_ss<T, 2, false>(pp, S, lamx, lamz, mean_out, st);
      if (n <= 128) return launch_ss<T, 4, false>(pp, S, lamx, lamz, mean_out, st);
      if (n <= 256) return launch_ss<T, 8, true>(pp, S, lamx, lamz, mean_out, st);
    } else {
      if (n <= 32) return launch_ss<T, 1, false>(pp, S, lamx, lamz, mean_out, st);
      if (n <= 64) return launch_ss<T, 2, false>(pp, S, lamx, lamz, mean_out, st);
      if (n <= 128) return launch_ss<T, 4, true>(pp, S, lamx, lamz, mean_out, st);
    }
  }
  constexpr int TP = PencilTile<T>::TP;
  const int npen = pp.nz * pp.P;
  const int grid = ceil_div(npen, TP) + (pp.zero_mode ? 1 : 0);
  const dim3 g2(grid, pp.nb);
  // the tile kernel while every CTA stays resident (measured faster there);
  // beyond that the tile-less kernel, which keeps about three times as many
  const size_t tb = pencil_smem_bytes<T>(pp.ny);
  const bool tile = pp.mode == 2 || (pp.mode != 3 && (long)grid * pp.nb <= resident_ctas(tb));
  if (tile) {
    cudaError_t e = ensure_max_smem<k_pencil<T>>();
    if (e != cudaSuccess) return e;
    IBM_KTRY(launch_pdl(k_pencil<T>, g2, 32, tb, st, S3, lamx, lamz, pp, mean_out));
  } else {
    cudaError_t e = ensure_max_smem<k_pencil_g<T>>();
    if (e != cudaSuccess) return e;
    IBM_KTRY(launch_pdl(k_pencil_g<T>, g2, 32, pencil_g_smem_bytes<T>(pp.ny), st, S3, lamx, lamz, pp, mean_out));
  }
  return cudaGetLastError();
}

template cudaError_t launch_pencil<float>(const PencilParams &, Ptr3<float2 *>, const float *, const float *,
                                          double *, cudaStream_t);
template cudaError_t launch_pencil<double>(const PencilParams &, Ptr3<double2 *>, const double *, const double *,
                                           double *, cudaStream_t);

}  // namespace ibm
