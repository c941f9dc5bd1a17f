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
#include "internal.h"
#include "tma.cuh"

namespace ibm {

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return rcp_approx(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

template <typename T> struct PencilTile { static constexpr int TP = 32; };
template <> struct PencilTile<double> { static constexpr int TP = 16; };

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
__device__ void zero_mode_fp64(const double *__restrict__ zrhs, double *__restrict__ zsol, double *zs, int ny,
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

// The extra CTA of a pencil grid: the FP64 zero mode (returns true if this
// CTA was that one).
__device__ __forceinline__ bool zero_mode_cta(const PencilParams &pp, double *zs, double *mean_out) {
  if (!pp.zero_mode || blockIdx.x != gridDim.x - 1) return false;
  if (threadIdx.x < 32)
    zero_mode_fp64(pp.zrhs, pp.zsol, zs, pp.ny, pp.inv_ny, pp.hy2, pp.inv_nxnz, mean_out);
  return true;
}

// One pencil per lane: Thomas in excess form on tile column `lane`.
template <typename T, int TP>
__device__ __forceinline__ void serial_sweep(cplx<T> *tile, T *qs, const T *__restrict__ lamx,
                                             const T *__restrict__ lamz, const PencilParams &pp, int p0, int lane,
                                             cplx<T> *__restrict__ col, size_t plane) {
  const int ny = pp.ny;

  const int p = p0 + lane;
  const int kz = p / pp.P, kx = p - kz * pp.P;
  const T a = (T)pp.a;
  const T g = (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]);
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const int j0 = pp.j0;
  const int n = ny - j0;
  cplx<T> *tl = tile + j0 * TP + lane;  // row i of the pencil at tl[i * TP]
  T *ql = qs + j0 * TP + lane;

  // forward sweep, rows 0 .. n-2 (y overwrites f in the tile, q kept for the way back)
  T e = g + a * (T)pp.beta_s;
  T r = rcp<T>(a + e);
  T q = e * r;
  cplx<T> y = tl[0];
  y.x = r * (sgn * y.x);
  y.y = r * (sgn * y.y);
  tl[0] = y;
  ql[0] = q;
#pragma unroll 4
  for (int i = 1; i < n - 1; ++i) {
    const cplx<T> f = tl[i * TP];
    e = fma(a, q, g);
    r = rcp<T>(a + e);
    q = e * r;
    y.x = fma(r, sgn * f.x, fma(-q, y.x, y.x));
    y.y = fma(r, sgn * f.y, fma(-q, y.y, y.y));
    tl[i * TP] = y;
    ql[i * TP] = q;
  }
  // last row: pivot a beta_e + e_{n-1}
  {
    const cplx<T> f = tl[(n - 1) * TP];
    e = fma(a, q, g);
    const T rl = rcp<T>(e + a * (T)pp.beta_e);
    y.x = (sgn * f.x + a * y.x) * rl;
    y.y = (sgn * f.y + a * y.y) * rl;
  }
  // backward sweep, results straight to global memory (fire-and-forget stores)
  cplx<T> *cj = col + (size_t)j0 * plane;
  cplx<T> x = y;
  cj[(size_t)(n - 1) * plane] = x;
  for (int i = n - 2; i >= 0; --i) {
    const T qi = ql[i * TP];
    const cplx<T> yi = tl[i * TP];
    x.x = fma(-qi, x.x, x.x) + yi.x;
    x.y = fma(-qi, x.y, x.y) + yi.y;
    cj[(size_t)i * plane] = x;
  }
  if (j0 == 1) {
    cplx<T> z; z.x = (T)0; z.y = (T)0;
    col[0] = z;
  }
}

template <typename T>
__global__ void __launch_bounds__(32)
k_pencil(cplx<T> *__restrict__ S, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
         double *mean_out) {
  constexpr int TP = PencilTile<T>::TP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw + 16);  // [ny][TP]
  T *qs = reinterpret_cast<T *>(tile + (size_t)pp.ny * TP);    // [ny][TP]
  double *zs = reinterpret_cast<double *>(qs + (size_t)pp.ny * TP);  // [ny]
  const int ny = pp.ny;
  if (zero_mode_cta(pp, zs, mean_out)) return;
  const size_t plane = (size_t)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int p0 = blockIdx.x * TP;
  const int np = min(TP, npen - p0);  // even: npen is even and p0 a multiple of TP
  const int lane = threadIdx.x;
  // one warp per CTA: rows j of the tile arrive by bulk copy (np * 8 or 16 bytes each)
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(cplx<T>) * np * ny));
  }
  __syncwarp();
  for (int j = lane; j < ny; j += 32)
    bulk_g2s(tile + (size_t)j * TP, S + (size_t)j * plane + p0, (uint32_t)(sizeof(cplx<T>) * np), bar);
  if (!__all_sync(0xffffffffu, mbar_wait(bar, 0, pp.err))) return;
  // the (0,0) pencil is singular (g = 0): its sweep is skipped here and its
  // FP64 solution reaches the inverse transform through zsol
  if (lane < np && !(pp.zero_mode && p0 == 0 && lane == 0))
    serial_sweep<T, TP>(tile, qs, lamx, lamz, pp, p0, lane, S + p0 + lane, plane);
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
  if (!__syncthreads_and(mbar_wait(bar, 0, pp.err))) return;


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
  k_pencil_ss<T, M, SPLIT><<<ceil_div(npen, C::TP) + (pp.zero_mode ? 1 : 0), 1024, bytes, st>>>(S, lamx, lamz, pp,
                                                                                             mean_out);
  return cudaGetLastError();
}

template <typename T> size_t pencil_smem_bytes(int ny) {
  constexpr int TP = PencilTile<T>::TP;
  return 16 + (size_t)ny * TP * (sizeof(cplx<T>) + sizeof(T)) + (size_t)ny * sizeof(double);
}

template <typename T>
cudaError_t launch_pencil(const PencilParams &pp, cplx<T> *S, const T *lamx, const T *lamz, double *mean_out,
                          cudaStream_t st) {
  const int n = pp.ny - pp.j0;
  if (pp.substructured) {
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
  const size_t bytes = pencil_smem_bytes<T>(pp.ny);
  {
    cudaError_t e = ensure_max_smem<k_pencil<T>>();
    if (e != cudaSuccess) return e;
  }
  const int npen = pp.nz * pp.P;
  k_pencil<T><<<ceil_div(npen, TP) + (pp.zero_mode ? 1 : 0), 32, bytes, st>>>(S, lamx, lamz, pp, mean_out);
  return cudaGetLastError();
}

template cudaError_t launch_pencil<float>(const PencilParams &, float2 *, const float *, const float *, double *,
                                          cudaStream_t);
template cudaError_t launch_pencil<double>(const PencilParams &, double2 *, const double *, const double *,
                                           double *, cudaStream_t);

}  // namespace ibm
