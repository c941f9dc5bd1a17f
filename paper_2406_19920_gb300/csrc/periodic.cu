// periodic.cu -- the pencil step of the triply periodic branch.
//
// With y periodic as well (Sec. 2.3.3, S2), every (kx, kz) pencil of the
// x/z spectrum is diagonalised by a Fourier transform along y too: the
// solve is a forward y-transform, a divide by the eigenvalue of each
// (kx, ky, kz) mode, and an inverse y-transform (scaled by 1/ny), all in
// place on the spectrum.  Eigenvalues (Appendix A): lambda = lambda_x(kx) +
// lambda_y(ky) + lambda_z(kz), lambda_d = (2/h_d^2)(1 - cos theta_d);
//   Poisson    x = -f / lambda, the (0,0,0) mode set to 0 (mean(phi) = 0);
//   Helmholtz  x =  f / (1 + c lambda).
// A CTA takes W consecutive pencils (every access a run of W complex
// values); both y-transforms are the two-step register FFT of fft2.cuh with
// one shared-memory exchange each, and the divided spectrum crosses shared
// memory once between them.  For the Poisson solve an extra CTA sums the
// FP64 plane sums of b (from the forward x/z transform) into the removed
// mean.
#include "fft2.cuh"
#include "internal.h"

namespace ibm {

template <typename T, int N> struct YCfg {
  static constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  static constexpr int WMIN = sizeof(T) == 4 ? 16 : 8, WMAX = 64;
  static constexpr int WT0 = 256 / N1;
  static constexpr int WS = (int)(32768 / ((size_t)N * sizeof(cplx<T>)));  // each of X, Y <= 32 KB
  static constexpr int WT = WT0 < WS ? WT0 : WS;
  static constexpr int W = WT < WMIN ? WMIN : (WT > WMAX ? WMAX : WT);
  static constexpr int THREADS = W * N1;
  static constexpr size_t smem = sizeof(cplx<T>) * ((size_t)N + 2 * (size_t)N * W);
};

template <typename T, int N>
__global__ void __launch_bounds__(YCfg<T, N>::THREADS)
k_ypencil(cplx<T> *__restrict__ S, const cplx<T> *__restrict__ tw, const T *__restrict__ lamx,
          const T *__restrict__ lamz, const T *__restrict__ lamy, PencilParams pp, double *mean_out) {
  using Cfg = YCfg<T, N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, W = Cfg::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2 = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *X = tw2 + N;      // [N1][N2][W] exchange of both transforms
  cplx<T> *Y = X + N * W;    // [N][W] divided y-spectrum
  load_step_twiddles<T, N>(tw2, tw);
  pdl_wait();
  if (pp.zero_mode && blockIdx.x == gridDim.x - 1) {
    // removed mean of b: the FP64 sum of the plane sums (zrhs) / (nx ny nz)
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int j = threadIdx.x; j < N; j += 32) s += pp.zrhs[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0 && mean_out) {
        const double m = s * pp.inv_nxnz * pp.inv_ny;
        mean_out[0] = m;
        float2 f;
        f.x = (float)m;
        f.y = (float)(m - (double)f.x);
        *reinterpret_cast<float2 *>(mean_out + 1) = f;
      }
    }
    return;
  }
  __syncthreads();
  const size_t plane = (size_t)pp.nz * pp.P;
  const int npen = pp.nz * pp.P;
  const int tid = threadIdx.x;
  const int c = tid % W;
  const int p = blockIdx.x * W + c;
  const bool live = p < npen;
  const int kz = live ? p / pp.P : 0, kx = live ? p - kz * pp.P : 0;
  cplx<T> *base = S + (live ? p : 0);
  const T lxz = lamx[kx] + lamz[kz];
  const T g_add = (T)pp.g_add, g_mul = (T)pp.g_mul;
  const T sgn = pp.neg_rhs ? (T)-1 : (T)1;
  const T inv_n = (T)1 / (T)N;
  // forward y-transform, step 1
  if (live) col_step1<T, N, false, W>(base, plane, tid / W, tw2, X + (tid / W) * N2 * W + c, false, mk<T>(0, 0));
  __syncthreads();
  // step 3 and the divide, into Y in natural ky order
  if (live) {
    for (int k2 = tid / W; k2 < N2; k2 += N1) {
      col_step3_at<T, N, false, W>(X, c, k2, [&](int a, int b) {
        const int ky = a + N2 * b;
        return Y + ky * W + c;
      });
    }
  }
  __syncthreads();
  if (live) {
    for (int ky = tid / W; ky < N; ky += N1) {
      const T eig = g_add + g_mul * (lxz + lamy[ky]);
      const cplx<T> f = Y[ky * W + c];
      const T s = eig != (T)0 ? sgn * inv_n / eig : (T)0;  // the (0,0,0) Poisson mode -> 0
      Y[ky * W + c] = mk<T>(f.x * s, f.y * s);
    }
  }
  __syncthreads();
  // inverse y-transform
  if (live)
    col_step1_at<T, N, true, W>([&](int a, int b) { return Y + (a + N1 * b) * W + c; }, tid / W, tw2,
                                X + (tid / W) * N2 * W + c, false, mk<T>(0, 0));
  __syncthreads();
  if (live)
    for (int k2 = tid / W; k2 < N2; k2 += N1) col_step3<T, N, true, W>(X, c, k2, base, plane);
}

#define IBM_Y_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

template <typename T>
cudaError_t launch_ypencil(const PencilParams &pp, Ptr3<cplx<T> *> S3, const cplx<T> *twy, const T *lamx,
                           const T *lamz, const T *lamy, double *mean_out, cudaStream_t st) {
  const int npen = pp.nz * pp.P;
  for (int b = 0; b < pp.nb; ++b) {
    bool done = false;
#define X(N)                                                                                      \
    if (pp.ny == N) {                                                                             \
      using Cfg = YCfg<T, N>;                                                                     \
      { cudaError_t e = ensure_max_smem<k_ypencil<T, N>>(); if (e) return e; }                   \
      const int grid = ceil_div(npen, Cfg::W) + (pp.zero_mode ? 1 : 0);                           \
      IBM_KTRY(launch_pdl(k_ypencil<T, N>, grid, Cfg::THREADS, Cfg::smem, st, S3[b], twy, lamx, lamz, lamy, pp, \
                          mean_out));                                                             \
      done = true;                                                                                \
    }
    IBM_Y_N(X)
#undef X
    if (!done) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

template cudaError_t launch_ypencil<float>(const PencilParams &, Ptr3<float2 *>, const float2 *, const float *,
                                           const float *, const float *, double *, cudaStream_t);
template cudaError_t launch_ypencil<double>(const PencilParams &, Ptr3<double2 *>, const double2 *, const double *,
                                            const double *, const double *, double *, cudaStream_t);

}  // namespace ibm
