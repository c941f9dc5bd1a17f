// axis.cu -- split transform passes: x rows, then z columns, each one kernel.
//
// Both passes use the two-step register transform (N = N1 x N2): step 1
// reads straight from global memory into the registers of N1 threads per
// row, step 3 writes straight back, and the one exchange in between goes
// through shared memory.  The spectrum between the two passes is the plan's
// spectrum array, which stays in the 129 MB L2 for grids up to ~256^3.
//
//   rows forward   real row pairs (a, b) -> z = a + i b -> Z; each step-3
//                  thread owns the columns k2 and N2 - k2, so it holds Z_k
//                  and Z_{N-k} together and writes the two half spectra
//                  A_k = (Z_k + conj Z_{N-k}) / 2, B_k = -i (Z_k - conj Z_{N-k}) / 2
//                  for k = 0..N/2 without a further exchange;
//   rows inverse   Z_k = A_k + i B_k (Hermitian extension, imaginary parts
//                  of the k = 0 and N/2 bins dropped) -> z; out = addend +
//                  scale (Re z, Im z) for the two rows;
//   columns        complex columns of stride P (= nx/2 + 1) in place; a CTA
//                  takes W consecutive columns of the flattened (plane, kx)
//                  list, threads along columns so that every global access
//                  is a run of W consecutive complex values.
#include "fft2.cuh"
#include "internal.h"

namespace ibm {

constexpr int kRowThreads = 256;

template <typename T, int N> struct RowCfg {
  static constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  static constexpr int RP = (kRowThreads / N1) > 1 ? kRowThreads / N1 : 1;  // row pairs per CTA
  static constexpr int PITCH = N2 + 1;                                      // odd: conflict-free exchange
  static constexpr size_t smem = sizeof(cplx<T>) * ((size_t)N + (size_t)RP * N1 * PITCH);
};

template <typename T, int N>
__global__ void __launch_bounds__(kRowThreads)
k_rows_fwd(Ptr3<const T *> in_, Ptr3<cplx<T> *> S_, const cplx<T> *__restrict__ tw, int npairs, T in_scale) {
  const T *__restrict__ in = in_[blockIdx.y];
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  using Cfg = RowCfg<T, N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, RP = Cfg::RP, PITCH = Cfg::PITCH, P = N / 2 + 1;
  constexpr int J3 = N2 / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2 = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *X = tw2 + N;  // [RP][N1][PITCH]
  load_step_twiddles<T, N>(tw2, tw);
  pdl_wait();  // the spectrum / fields below are the predecessor's output
  const int pair0 = blockIdx.x * RP;
  const int np = min(RP, npairs - pair0);
  __syncthreads();
  for (int job = threadIdx.x; job < np * N1; job += kRowThreads) {
    const int p = job / N1, n1 = job - p * N1;
    rfwd_step1<T, N>(in + (size_t)(pair0 + p) * 2 * N, in_scale, n1, tw2, X + (p * N1 + n1) * PITCH);
  }
  __syncthreads();
  for (int job = threadIdx.x; job < np * J3; job += kRowThreads) {
    const int p = job / J3, q = job - p * J3;
    cplx<T> *dA = S + (size_t)(pair0 + p) * 2 * P;
    rfwd_step3<T, N, PITCH>(X + p * N1 * PITCH, q, dA, dA + P);
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(kRowThreads)
k_rows_inv(Ptr3<cplx<T> *> S_, Ptr3<T *> out_, Ptr3<const T *> add_, const cplx<T> *__restrict__ tw, int npairs,
           T scale) {
  const cplx<T> *__restrict__ S = S_[blockIdx.y];
  T *out = out_[blockIdx.y];
  const T *addend = add_[blockIdx.y];
  using Cfg = RowCfg<T, N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, RP = Cfg::RP, PITCH = Cfg::PITCH, P = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2 = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *X = tw2 + N;
  load_step_twiddles<T, N>(tw2, tw);
  pdl_wait();  // the spectrum / fields below are the predecessor's output
  const int pair0 = blockIdx.x * RP;
  const int np = min(RP, npairs - pair0);
  __syncthreads();
  for (int job = threadIdx.x; job < np * N1; job += kRowThreads) {
    const int p = job / N1, n1 = job - p * N1;
    const cplx<T> *sA = S + (size_t)(pair0 + p) * 2 * P;
    rinv_step1<T, N>(sA, sA + P, n1, tw2, X + (p * N1 + n1) * PITCH);
  }
  __syncthreads();
  for (int job = threadIdx.x; job < np * N2; job += kRowThreads) {
    const int p = job / N2, k2 = job - p * N2;
    T *da = out + (size_t)(pair0 + p) * 2 * N;
    const T *aa = addend ? addend + (size_t)(pair0 + p) * 2 * N : nullptr;
    rinv_step3<T, N, PITCH>(X + p * N1 * PITCH, k2, da, da + N, aa, aa ? aa + N : nullptr, scale);
  }
}

template <typename T, int N> struct ColCfg {
  static constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  // columns per CTA: runs of >= 128 bytes per row; one thread per (column,
  // n1) in step 1, and the same threads take the N2 step-3 DFTs of their
  // column in turn (about 256 threads, every one busy in both steps)
  static constexpr int WMIN = sizeof(T) == 4 ? 16 : 8, WMAX = 64;
  static constexpr int WT0 = 256 / N1;
  static constexpr int WS = (int)(65536 / ((size_t)N * sizeof(cplx<T>)));  // exchange tile <= 64 KB
  static constexpr int WT = WT0 < WS ? WT0 : WS;
  static constexpr int W = WT < WMIN ? WMIN : (WT > WMAX ? WMAX : WT);
  static constexpr int THREADS = W * N1;
  static constexpr size_t smem = sizeof(cplx<T>) * ((size_t)N + (size_t)N * W);
};

// z columns in place.  Column `col` of the flattened list is kx = col % P of
// plane j = col / P; element kz at S[(j NZ + kz) P + kx].
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(ColCfg<T, N>::THREADS)
k_cols(Ptr3<cplx<T> *> S_, const cplx<T> *__restrict__ tw, int P, int ncols, double *zrhs, const double *zsol) {
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  using Cfg = ColCfg<T, N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, W = Cfg::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2 = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *X = tw2 + N;  // [N1][N2][W]
  load_step_twiddles<T, N>(tw2, tw);
  pdl_wait();  // the spectrum / fields below are the predecessor's output
  __syncthreads();
  const int tid = threadIdx.x;
  const int c = tid % W;
  const int col = blockIdx.x * W + c;
  const bool live = col < ncols;
  const int j = live ? col / P : 0;
  const int kx = live ? col - j * P : 0;
  cplx<T> *base = S + (size_t)j * N * P + kx;
  if (live) {
    const int n1 = tid / W;
    const bool sub = INV && zsol && kx == 0;
    col_step1<T, N, INV, W>(base, P, n1, tw2, X + n1 * N2 * W + c, sub,
                            sub ? mk<T>((T)zsol[j], (T)0) : mk<T>((T)0, (T)0));
  }
  __syncthreads();
  if (live) {
    for (int k2 = tid / W; k2 < N2; k2 += N1) {
      const cplx<T> u0 = col_step3<T, N, INV, W>(X, c, k2, base, P);
      if (!INV && zrhs && kx == 0 && k2 == 0) zrhs[j] = (double)u0.x;
    }
  }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
#define IBM_AXIS_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

template <typename T>
cudaError_t launch_axis_forward(const TransformGeom &g, Ptr3<const T *> in, Ptr3<cplx<T> *> S, const cplx<T> *twx,
                                const cplx<T> *twz, T in_scale, cudaStream_t st) {
  const int npairs = g.ny * g.nz / 2;
  const int P = g.nx / 2 + 1;
  bool done = false;
#define X(N)                                                                                      \
  if (g.nx == N) {                                                                                \
    using Cfg = RowCfg<T, N>;                                                                     \
    { cudaError_t e = ensure_max_smem<k_rows_fwd<T, N>>(); if (e) return e; }                     \
    IBM_KTRY(launch_pdl(k_rows_fwd<T, N>, dim3(ceil_div(npairs, Cfg::RP), g.nb), kRowThreads, Cfg::smem, st, in, S, twx, npairs, in_scale)); \
    done = true;                                                                                  \
  }
  IBM_AXIS_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  done = false;
  const int ncols = g.ny * P;
#define X(N)                                                                                      \
  if (g.nz == N) {                                                                                \
    using Cfg = ColCfg<T, N>;                                                                     \
    { cudaError_t e = ensure_max_smem<k_cols<T, N, false>>(); if (e) return e; }                  \
    IBM_KTRY(launch_pdl(k_cols<T, N, false>, dim3(ceil_div(ncols, Cfg::W), g.nb), Cfg::THREADS, Cfg::smem, st, S, twz, P, ncols, g.zrhs, nullptr)); \
    done = true;                                                                                  \
  }
  IBM_AXIS_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axis_inverse(const TransformGeom &g, Ptr3<cplx<T> *> S, Ptr3<T *> out, Ptr3<const T *> addend,
                                const cplx<T> *twx, const cplx<T> *twz, T scale, cudaStream_t st) {
  const int npairs = g.ny * g.nz / 2;
  const int P = g.nx / 2 + 1;
  const int ncols = g.ny * P;
  bool done = false;
#define X(N)                                                                                      \
  if (g.nz == N) {                                                                                \
    using Cfg = ColCfg<T, N>;                                                                     \
    { cudaError_t e = ensure_max_smem<k_cols<T, N, true>>(); if (e) return e; }                   \
    IBM_KTRY(launch_pdl(k_cols<T, N, true>, dim3(ceil_div(ncols, Cfg::W), g.nb), Cfg::THREADS, Cfg::smem, st, S, twz, P, ncols, nullptr, g.zsol)); \
    done = true;                                                                                  \
  }
  IBM_AXIS_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  done = false;
#define X(N)                                                                                      \
  if (g.nx == N) {                                                                                \
    using Cfg = RowCfg<T, N>;                                                                     \
    { cudaError_t e = ensure_max_smem<k_rows_inv<T, N>>(); if (e) return e; }                     \
    IBM_KTRY(launch_pdl(k_rows_inv<T, N>, dim3(ceil_div(npairs, Cfg::RP), g.nb), kRowThreads, Cfg::smem, st, S, out, addend, twx, npairs, scale)); \
    done = true;                                                                                  \
  }
  IBM_AXIS_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template cudaError_t launch_axis_forward<float>(const TransformGeom &, Ptr3<const float *>, Ptr3<float2 *>,
                                                const float2 *, const float2 *, float, cudaStream_t);
template cudaError_t launch_axis_forward<double>(const TransformGeom &, Ptr3<const double *>, Ptr3<double2 *>,
                                                 const double2 *, const double2 *, double, cudaStream_t);
template cudaError_t launch_axis_inverse<float>(const TransformGeom &, Ptr3<float2 *>, Ptr3<float *>,
                                                Ptr3<const float *>, const float2 *, const float2 *, float,
                                                cudaStream_t);
template cudaError_t launch_axis_inverse<double>(const TransformGeom &, Ptr3<double2 *>, Ptr3<double *>,
                                                 Ptr3<const double *>, const double2 *, const double2 *, double,
                                                 cudaStream_t);

}  // namespace ibm
