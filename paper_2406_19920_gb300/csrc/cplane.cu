// cplane.cu -- plane transforms by a thread-block cluster of C CTAs per y-plane.
//
// For planes whose spectrum does not fit one CTA's shared memory (256^2 and
// larger in FP32).  CTA r of the cluster owns the z-rows [r R, (r+1) R)
// (R = NZ/C) of the plane's half spectrum in its shared memory and the kx
// columns [r Pc, (r+1) Pc) (Pc = ceil(P/C), P = NX/2+1):
//   forward  x-transform of its row pairs straight from HBM into its rows
//            (two-step register FFT, fft2.cuh); cluster barrier; z-transform
//            of its columns, step 1 reading each column element from the CTA
//            that owns the row (distributed shared memory), step 3 writing
//            straight to HBM; cluster barrier (peers still read its rows);
//   inverse  z-transform of its columns straight from HBM, step 3 writing
//            each element into the owner CTA's rows (distributed shared
//            memory); cluster barrier; x-inverse of its own row pairs with the
//            addend, straight to HBM.
// The transpose between the two transform directions happens in shared
// memory across the cluster; each element crosses HBM once per direction.
// Every CTA reaches every cluster barrier.
#include <cooperative_groups.h>

#include "fft2.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace ibm {

template <typename T, int NX, int NZ, int C> struct ClusterCfg {
  using Cx = cplx<T>;
  static constexpr int P = NX / 2 + 1;
  static constexpr int R = NZ / C;                // z-rows per CTA
  static constexpr int PC = (P + C - 1) / C;      // kx columns per CTA
  static constexpr int N1X = TwoStep<NX>::N1, N2X = TwoStep<NX>::N2, XPITCH = N2X + 1;
  static constexpr int N1Z = TwoStep<NZ>::N1, N2Z = TwoStep<NZ>::N2;
  static constexpr size_t fixed = sizeof(Cx) * ((size_t)NX + NZ + (size_t)R * P);
  static constexpr size_t room = fixed < kPlaneSmemLimit ? kPlaneSmemLimit - fixed : 0;
  static constexpr size_t pair_bytes = sizeof(Cx) * N1X * XPITCH;
  static constexpr size_t col_bytes = sizeof(Cx) * NZ;
  static constexpr int CP0 = (int)(room / pair_bytes), CW0 = (int)(room / col_bytes);
  static constexpr int CP = CP0 < R / 2 ? CP0 : R / 2;  // row pairs per x chunk
  static constexpr int CW = CW0 < PC ? CW0 : PC;        // columns per z chunk
  // a column's element n1 + N1z n2 lives in CTA n2 / (R / N1z) (R a multiple of N1z and N2z)
  static constexpr bool ok = R % 2 == 0 && R % N1Z == 0 && R % N2Z == 0 && CP >= 4 && CW >= 4;
  static constexpr size_t xbytes = (size_t)CP * pair_bytes > (size_t)CW * col_bytes ? (size_t)CP * pair_bytes
                                                                                    : (size_t)CW * col_bytes;
  static constexpr size_t bytes = fixed + xbytes;
  static constexpr int J3 = N2X / 2 + 1;
  static constexpr int JMAX0 = CP * N1X > CP * J3 ? CP * N1X : CP * J3;
  static constexpr int JMAX = JMAX0 > CW * N1Z ? JMAX0 : CW * N1Z;
  static constexpr int THREADS = JMAX >= 1024 ? 1024 : (JMAX + 31) / 32 * 32;
};

template <typename T, int NX, int NZ, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(ClusterCfg<T, NX, NZ, C>::THREADS)
k_cplane_fwd(Ptr3<const T *> in_, Ptr3<cplx<T> *> S_, const cplx<T> *__restrict__ twx,
             const cplx<T> *__restrict__ twz, T in_scale, double *zrhs) {
  using Cfg = ClusterCfg<T, NX, NZ, C>;
  constexpr int P = Cfg::P, R = Cfg::R, PC = Cfg::PC, N1X = Cfg::N1X, XPITCH = Cfg::XPITCH;
  constexpr int N1Z = Cfg::N1Z, N2Z = Cfg::N2Z, CP = Cfg::CP, CW = Cfg::CW, J3 = Cfg::J3, NT = Cfg::THREADS;
  constexpr int RB = R / N1Z;  // n2 values per owner CTA
  const T *__restrict__ in = in_[blockIdx.y];
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int j = blockIdx.x / C;
  const int tid = threadIdx.x;
  cplx<T> *tw2x = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *tw2z = tw2x + NX;
  cplx<T> *hp = tw2z + NZ;  // [R][P]: this CTA's rows of the plane's half spectrum
  cplx<T> *X = hp + R * P;
  load_step_twiddles<T, NX>(tw2x, twx);
  load_step_twiddles<T, NZ>(tw2z, twz);
  pdl_wait();
  __syncthreads();
  // x: own row pairs -> own rows of hp
  const T *src = in + ((size_t)j * NZ + (size_t)r * R) * NX;
  for (int p0 = 0; p0 < R / 2; p0 += CP) {
    const int np = min(CP, R / 2 - p0);
    for (int job = tid; job < np * N1X; job += NT) {
      const int p = job / N1X, n1 = job - p * N1X;
      rfwd_step1<T, NX>(src + (size_t)(p0 + p) * 2 * NX, in_scale, n1, tw2x, X + (p * N1X + n1) * XPITCH);
    }
    __syncthreads();
    for (int job = tid; job < np * J3; job += NT) {
      const int p = job / J3, q = job - p * J3;
      cplx<T> *dA = hp + (p0 + p) * 2 * P;
      rfwd_step3<T, NX, XPITCH>(X + p * N1X * XPITCH, q, dA, dA + P);
    }
    __syncthreads();
  }
  cluster.sync();
  // z: own columns, elements from the owner CTAs' rows
  const cplx<T> *rows[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rows[q] = cluster.map_shared_rank(hp, q);
  const int cbeg = r * PC, cend = min(P, cbeg + PC);
  cplx<T> *dst = S + (size_t)j * NZ * P;
  for (int c0 = cbeg; c0 < cend; c0 += CW) {
    const int nc = min(CW, cend - c0);
    for (int job = tid; job < CW * N1Z; job += NT) {
      const int n1 = job / CW, c = job - n1 * CW;
      if (c < nc) {
        const int kx = c0 + c;
        col_step1_at<T, NZ, false, CW>(
            [&](int a, int b) { return rows[b / RB] + (a + N1Z * (b % RB)) * P + kx; }, n1, tw2z,
            X + n1 * N2Z * CW + c, false, mk<T>((T)0, (T)0));
      }
    }
    __syncthreads();
    for (int job = tid; job < CW * N2Z; job += NT) {
      const int k2 = job / CW, c = job - k2 * CW;
      if (c < nc) {
        const cplx<T> u0 = col_step3<T, NZ, false, CW>(X, c, k2, dst + c0 + c, P);
        if (zrhs && c0 + c == 0 && k2 == 0) zrhs[j] = (double)u0.x;
      }
    }
    __syncthreads();
  }
  cluster.sync();  // peers are done reading this CTA's rows
}

template <typename T, int NX, int NZ, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(ClusterCfg<T, NX, NZ, C>::THREADS)
k_cplane_inv(Ptr3<cplx<T> *> S_, Ptr3<T *> out_, Ptr3<const T *> add_, const cplx<T> *__restrict__ twx,
             const cplx<T> *__restrict__ twz, T scale, const double *zsol) {
  using Cfg = ClusterCfg<T, NX, NZ, C>;
  constexpr int P = Cfg::P, R = Cfg::R, PC = Cfg::PC, N1X = Cfg::N1X, N2X = Cfg::N2X, XPITCH = Cfg::XPITCH;
  constexpr int N1Z = Cfg::N1Z, N2Z = Cfg::N2Z, CP = Cfg::CP, CW = Cfg::CW, NT = Cfg::THREADS;
  constexpr int RB = R / N2Z;  // k1 values per owner CTA
  const cplx<T> *__restrict__ S = S_[blockIdx.y];
  T *out = out_[blockIdx.y];
  const T *addend = add_[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int j = blockIdx.x / C;
  const int tid = threadIdx.x;
  cplx<T> *tw2x = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *tw2z = tw2x + NX;
  cplx<T> *hp = tw2z + NZ;
  cplx<T> *X = hp + R * P;
  load_step_twiddles<T, NX>(tw2x, twx);
  load_step_twiddles<T, NZ>(tw2z, twz);
  pdl_wait();
  __syncthreads();
  cplx<T> *rows[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rows[q] = cluster.map_shared_rank(hp, q);
  // every CTA's hp is live before any peer writes into it
  cluster.sync();
  // z: own columns from HBM, results into the owner CTAs' rows
  const cplx<T> *srcS = S + (size_t)j * NZ * P;
  const cplx<T> z0 = zsol ? mk<T>((T)zsol[j], (T)0) : mk<T>((T)0, (T)0);
  const int cbeg = r * PC, cend = min(P, cbeg + PC);
  for (int c0 = cbeg; c0 < cend; c0 += CW) {
    const int nc = min(CW, cend - c0);
    for (int job = tid; job < CW * N1Z; job += NT) {
      const int n1 = job / CW, c = job - n1 * CW;
      if (c < nc)
        col_step1<T, NZ, true, CW>(srcS + c0 + c, P, n1, tw2z, X + n1 * N2Z * CW + c, zsol && c0 + c == 0, z0);
    }
    __syncthreads();
    for (int job = tid; job < CW * N2Z; job += NT) {
      const int k2 = job / CW, c = job - k2 * CW;
      if (c < nc) {
        const int kx = c0 + c;
        col_step3_at<T, NZ, true, CW>(X, c, k2,
                                      [&](int a, int b) { return rows[b / RB] + (a + N2Z * (b % RB)) * P + kx; });
      }
    }
    __syncthreads();
  }
  cluster.sync();  // all of this CTA's rows have arrived
  // x: own row pairs from hp, with the addend, to HBM
  const size_t row0 = ((size_t)j * NZ + (size_t)r * R) * NX;
  T *dst = out + row0;
  const T *add = addend ? addend + row0 : nullptr;
  for (int p0 = 0; p0 < R / 2; p0 += CP) {
    const int np = min(CP, R / 2 - p0);
    for (int job = tid; job < np * N1X; job += NT) {
      const int p = job / N1X, n1 = job - p * N1X;
      const cplx<T> *sA = hp + (p0 + p) * 2 * P;
      rinv_step1<T, NX>(sA, sA + P, n1, tw2x, X + (p * N1X + n1) * XPITCH);
    }
    __syncthreads();
    for (int job = tid; job < np * N2X; job += NT) {
      const int p = job / N2X, k2 = job - p * N2X;
      const size_t rr = (size_t)(p0 + p) * 2 * NX;
      rinv_step3<T, NX, XPITCH>(X + p * N1X * XPITCH, k2, dst + rr, dst + rr + NX, add ? add + rr : nullptr,
                                add ? add + rr + NX : nullptr, scale);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// dispatch: shapes x cluster sizes instantiated here
// ---------------------------------------------------------------------------
#define IBM_CPLANE_CASES(X)                                                                     \
  X(64, 64, 2) X(96, 96, 2) X(128, 128, 2) X(192, 192, 2) X(256, 256, 2) X(256, 256, 4)        \
  X(256, 128, 2) X(128, 256, 2)                                                                 \
  X(384, 256, 4) X(384, 384, 4) X(512, 256, 4) X(512, 512, 8) X(384, 384, 8)

template <typename T> bool cplane_supported(int nx, int nz, int C) {
#define X(a, b, c) if (nx == a && nz == b && C == c) return ClusterCfg<T, a, b, c>::ok;
  IBM_CPLANE_CASES(X)
#undef X
  return false;
}

template <typename T>
cudaError_t launch_cplane_forward(const TransformGeom &g, int C, Ptr3<const T *> in, Ptr3<cplx<T> *> S,
                                  const cplx<T> *twx, const cplx<T> *twz, T in_scale, cudaStream_t st) {
#define X(a, b, c)                                                                              \
  if (g.nx == a && g.nz == b && C == c) {                                                       \
    if constexpr (ClusterCfg<T, a, b, c>::ok) {                                                 \
      using Cfg = ClusterCfg<T, a, b, c>;                                                       \
      { cudaError_t e = ensure_max_smem<k_cplane_fwd<T, a, b, c>>(); if (e) return e; }          \
      IBM_KTRY(launch_pdl(k_cplane_fwd<T, a, b, c>, dim3(g.ny * c, g.nb), Cfg::THREADS, Cfg::bytes, st, in, S, \
                          twx, twz, in_scale, g.zrhs));                                         \
      return cudaSuccess;                                                                       \
    }                                                                                           \
  }
  IBM_CPLANE_CASES(X)
#undef X
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_cplane_inverse(const TransformGeom &g, int C, Ptr3<cplx<T> *> S, Ptr3<T *> out,
                                  Ptr3<const T *> addend, const cplx<T> *twx, const cplx<T> *twz, T scale,
                                  cudaStream_t st) {
#define X(a, b, c)                                                                              \
  if (g.nx == a && g.nz == b && C == c) {                                                       \
    if constexpr (ClusterCfg<T, a, b, c>::ok) {                                                 \
      using Cfg = ClusterCfg<T, a, b, c>;                                                       \
      { cudaError_t e = ensure_max_smem<k_cplane_inv<T, a, b, c>>(); if (e) return e; }          \
      IBM_KTRY(launch_pdl(k_cplane_inv<T, a, b, c>, dim3(g.ny * c, g.nb), Cfg::THREADS, Cfg::bytes, st, S, out, \
                          addend, twx, twz, scale, g.zsol));                                    \
      return cudaSuccess;                                                                       \
    }                                                                                           \
  }
  IBM_CPLANE_CASES(X)
#undef X
  return cudaErrorNotSupported;
}

template bool cplane_supported<float>(int, int, int);
template bool cplane_supported<double>(int, int, int);
template cudaError_t launch_cplane_forward<float>(const TransformGeom &, int, Ptr3<const float *>, Ptr3<float2 *>,
                                                  const float2 *, const float2 *, float, cudaStream_t);
template cudaError_t launch_cplane_forward<double>(const TransformGeom &, int, Ptr3<const double *>,
                                                   Ptr3<double2 *>, const double2 *, const double2 *, double,
                                                   cudaStream_t);
template cudaError_t launch_cplane_inverse<float>(const TransformGeom &, int, Ptr3<float2 *>, Ptr3<float *>,
                                                  Ptr3<const float *>, const float2 *, const float2 *, float,
                                                  cudaStream_t);
template cudaError_t launch_cplane_inverse<double>(const TransformGeom &, int, Ptr3<double2 *>, Ptr3<double *>,
                                                   Ptr3<const double *>, const double2 *, const double2 *, double,
                                                   cudaStream_t);

}  // namespace ibm
