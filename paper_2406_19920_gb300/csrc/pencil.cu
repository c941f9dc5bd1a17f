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
// solved in FP64: the right-hand side is made compatible by removing its mean
// (reported as the removed mean of b), the paper's pin x_0 = 0 fixes the
// constant (Sec. 2.3.3, S2.1), the bidiagonal factors of the zero-mode matrix
// reduce the elimination to two running sums (a (x_{j+1} - x_j) =
// sum_{i<=j} f_i), and the FP64 mean of x is removed (mean(phi) = 0).
#include "internal.h"

namespace ibm {

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
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

// FP64 zero-mode pencil by one full warp.  f_j = Re(tile[j*TP]).
template <typename T>
__device__ void zero_mode_fp64(const cplx<T> *tile, int TP, double *zs, int ny, double hy2, double inv_nxnz,
                               cplx<T> *S, size_t plane, double *mean_out) {
  const int lane = threadIdx.x & 31;
  const int c = (ny + 31) / 32;
  const int lo = min(ny, lane * c), hi = min(ny, lo + c);
  double s = 0.0;
  for (int j = lo; j < hi; ++j) {
    const double v = (double)tile[j * TP].x;
    zs[j] = v;
    s += v;
  }
  const double mean = warp_sum(s) / ny;
  if (lane == 0 && mean_out) *mean_out = mean * inv_nxnz;
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
  const double m2 = warp_sum(s2) / ny;
  for (int j = lo; j < hi; ++j) {
    cplx<T> o; o.x = (T)(zs[j] - m2); o.y = (T)0;
    S[(size_t)j * plane] = o;
  }
}

template <typename T>
__global__ void __launch_bounds__(128)
k_pencil(cplx<T> *__restrict__ S, const T *__restrict__ lamx, const T *__restrict__ lamz, PencilParams pp,
         double *mean_out) {
  constexpr int TP = PencilTile<T>::TP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw);      // [ny][TP]
  T *qs = reinterpret_cast<T *>(tile + (size_t)pp.ny * TP);    // [ny][TP]
  double *zs = reinterpret_cast<double *>(qs + (size_t)pp.ny * TP + (TP & 1));  // [ny]
  const int ny = pp.ny;
  const size_t plane = (size_t)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int p0 = blockIdx.x * TP;
  const int np = min(TP, npen - p0);
  for (int idx = threadIdx.x; idx < ny * TP; idx += blockDim.x) {
    const int j = idx / TP, t = idx - j * TP;
    if (t < np) tile[idx] = S[(size_t)j * plane + p0 + t];
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const bool zero = pp.zero_mode && p0 == 0;
  if (zero) zero_mode_fp64<T>(tile, TP, zs, ny, pp.hy2, pp.inv_nxnz, S, plane, mean_out);
  if (lane >= np || (zero && lane == 0)) return;

  const int p = p0 + lane;
  const int kz = p / pp.P, kx = p - kz * pp.P;
  const T a = (T)pp.a;
  const T g = (T)pp.g_add + (T)pp.g_mul * (lamx[kx] + lamz[kz]);
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const int j0 = pp.j0;
  const int n = ny - j0;
  cplx<T> *col = S + p;
  cplx<T> *tl = tile + lane;
  T *ql = qs + lane;

  // forward sweep, rows 0 .. n-2
  T e = g + a * (T)pp.beta_s;
  T r = rcp<T>(a + e);
  T q = e * r;
  cplx<T> f = tl[(size_t)j0 * TP];
  cplx<T> y;
  y.x = r * (sgn * f.x);
  y.y = r * (sgn * f.y);
  tl[(size_t)j0 * TP] = y;
  ql[(size_t)j0 * TP] = q;
  for (int i = 1; i < n - 1; ++i) {
    const int jj = (j0 + i) * TP;
    e = g + a * q;
    r = rcp<T>(a + e);
    q = e * r;
    f = tl[jj];
    y.x = fma(r, sgn * f.x, fma(-q, y.x, y.x));
    y.y = fma(r, sgn * f.y, fma(-q, y.y, y.y));
    tl[jj] = y;
    ql[jj] = q;
  }
  // last row: pivot a beta_e + e_{n-1}
  {
    const int jj = (j0 + n - 1) * TP;
    e = g + a * q;
    const T rl = rcp<T>(e + a * (T)pp.beta_e);
    f = tl[jj];
    y.x = (sgn * f.x + a * y.x) * rl;
    y.y = (sgn * f.y + a * y.y) * rl;
  }
  // backward sweep
  cplx<T> x = y;
  col[(size_t)(j0 + n - 1) * plane] = x;
  for (int i = n - 2; i >= 0; --i) {
    const int jj = (j0 + i) * TP;
    const T qi = ql[jj];
    const cplx<T> yi = tl[jj];
    x.x = fma(-qi, x.x, x.x) + yi.x;
    x.y = fma(-qi, x.y, x.y) + yi.y;
    col[(size_t)(j0 + i) * plane] = x;
  }
  if (j0 == 1) {
    cplx<T> z; z.x = (T)0; z.y = (T)0;
    col[0] = z;
  }
}

template <typename T> size_t pencil_smem_bytes(int ny) {
  constexpr int TP = PencilTile<T>::TP;
  return (size_t)ny * TP * (sizeof(cplx<T>) + sizeof(T)) + sizeof(T) * 2 + (size_t)ny * sizeof(double) + 16;
}

template <typename T>
cudaError_t launch_pencil(const PencilParams &pp, cplx<T> *S, const T *lamx, const T *lamz, double *mean_out,
                          cudaStream_t st) {
  constexpr int TP = PencilTile<T>::TP;
  const size_t bytes = pencil_smem_bytes<T>(pp.ny);
  static size_t attr_bytes = 0;
  if (bytes > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_pencil<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    attr_bytes = bytes;
  }
  const int npen = pp.nz * pp.P;
  k_pencil<T><<<ceil_div(npen, TP), 128, bytes, st>>>(S, lamx, lamz, pp, mean_out);
  return cudaGetLastError();
}

template cudaError_t launch_pencil<float>(const PencilParams &, float2 *, const float *, const float *, double *,
                                          cudaStream_t);
template cudaError_t launch_pencil<double>(const PencilParams &, double2 *, const double *, const double *,
                                           double *, cudaStream_t);

}  // namespace ibm
