// transforms.cu -- Fourier transforms along the two periodic axes (x, z).
//
// The paper's doubly periodic branch (Sec. 2.3.3, S1.1/S2.1) feeds the
// pencil solver with the 2-D real FFT of the right-hand side over the
// periodic planes and inverts it afterwards (S1.2/S2.2).  Here each y-plane
// [nz][nx] (real) maps to a spectrum plane [nz][nx/2+1] (complex, kx
// fastest), unnormalised forward and scaled by 1/(nx nz) on the way back.
//
// Real rows are transformed in pairs: rows a and b form z = a + i b, one
// complex FFT of length nx gives Z, and A_k = (Z_k + conj Z_{N-k})/2,
// B_k = -i (Z_k - conj Z_{N-k})/2 for k = 0..nx/2.  The inverse rebuilds
// Z_k = A_k + i B_k from the two Hermitian half spectra.
//
// Three kernel families, chosen per plan by its plane mode:
//   plane kernels   (mode 1, here) one CTA per y-plane: the x transform of
//                   every row pair lands in a shared-memory plane, the z
//                   transform of every column leaves it; one HBM read and
//                   one write per direction;
//   axis kernels    (mode 0, axis.cu) x-rows and z-columns in two passes;
//   cluster kernels (modes 2, 4, 8, cplane.cu) C CTAs per plane.
// Plane and axis kernels run the two-step register transform of fft2.cuh.
#include "fft2.cuh"
#include "internal.h"

namespace ibm {

// --------------------------------------------------------------------------
// plane kernels: one CTA per y-plane
// --------------------------------------------------------------------------
// Shared memory (complex entries): tw2x [NX], tw2z [NZ], the spectrum plane
// [NZ][P], and one exchange buffer reused by the x chunks (CP row pairs,
// [CP][N1x][N2x+1]) and the z chunks (CW columns, [N1z][N2z][CW]); chunk
// sizes fill what the plane leaves of the 227 KB.
template <typename T, int NX, int NZ> struct PlaneCfg {
  using C = cplx<T>;
  static constexpr int P = NX / 2 + 1;
  static constexpr int N1X = TwoStep<NX>::N1, N2X = TwoStep<NX>::N2, XPITCH = N2X + 1;
  static constexpr size_t fixed = sizeof(C) * ((size_t)NX + NZ + (size_t)NZ * P);
  static constexpr size_t room = fixed < kPlaneSmemLimit ? kPlaneSmemLimit - fixed : 0;
  static constexpr size_t pair_bytes = sizeof(C) * N1X * XPITCH;
  static constexpr size_t col_bytes = sizeof(C) * NZ;
  static constexpr int CP0 = (int)(room / pair_bytes), CW0 = (int)(room / col_bytes);
  static constexpr int CP = CP0 < NZ / 2 ? CP0 : NZ / 2;
  static constexpr int CW = CW0 < P ? CW0 : P;
  static constexpr bool ok = CP >= (NZ / 2 < 8 ? NZ / 2 : 8) && CW >= (P < 8 ? P : 8);
  static constexpr size_t xbytes = (size_t)CP * pair_bytes > (size_t)CW * col_bytes ? (size_t)CP * pair_bytes
                                                                                    : (size_t)CW * col_bytes;
  static constexpr size_t bytes = fixed + xbytes;
  // threads: enough for the largest of the x step-1, x step-3 and z step-1
  // job counts in one round (z step 3 takes N2z / N1z rounds), <= 1024
  static constexpr int N1Z = TwoStep<NZ>::N1;
  static constexpr int J3 = N2X / 2 + 1;
  static constexpr int JMAX0 = CP * N1X > CP * J3 ? CP * N1X : CP * J3;
  static constexpr int JMAX = JMAX0 > CW * N1Z ? JMAX0 : CW * N1Z;
  static constexpr int THREADS = JMAX >= 1024 ? 1024 : (JMAX + 31) / 32 * 32;
};

template <typename T, int NX, int NZ>
__global__ void __launch_bounds__(PlaneCfg<T, NX, NZ>::THREADS)
k_plane_fwd(Ptr3<const T *> in_, Ptr3<cplx<T> *> S_, const cplx<T> *__restrict__ twx,
            const cplx<T> *__restrict__ twz, T in_scale, double *zrhs) {
  const T *__restrict__ in = in_[blockIdx.y];
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  using Cfg = PlaneCfg<T, NX, NZ>;
  constexpr int P = Cfg::P, N1X = Cfg::N1X, XPITCH = Cfg::XPITCH, CP = Cfg::CP, CW = Cfg::CW;
  constexpr int kPlaneThreads_ = Cfg::THREADS;
  constexpr int N1Z = TwoStep<NZ>::N1, N2Z = TwoStep<NZ>::N2, J3 = Cfg::N2X / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2x = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *tw2z = tw2x + NX;
  cplx<T> *plane = tw2z + NZ;  // [NZ][P]
  cplx<T> *X = plane + NZ * P;
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  load_step_twiddles<T, NX>(tw2x, twx);
  load_step_twiddles<T, NZ>(tw2z, twz);
  pdl_wait();  // the fields below are the predecessor's output
  __syncthreads();
  const T *src = in + (size_t)j * NZ * NX;
  for (int p0 = 0; p0 < NZ / 2; p0 += CP) {
    const int np = min(CP, NZ / 2 - p0);
    for (int job = tid; job < np * N1X; job += kPlaneThreads_) {
      const int p = job / N1X, n1 = job - p * N1X;
      rfwd_step1<T, NX>(src + (size_t)(p0 + p) * 2 * NX, in_scale, n1, tw2x, X + (p * N1X + n1) * XPITCH);
    }
    __syncthreads();
    for (int job = tid; job < np * J3; job += kPlaneThreads_) {
      const int p = job / J3, q = job - p * J3;
      cplx<T> *dA = plane + (p0 + p) * 2 * P;
      rfwd_step3<T, NX, XPITCH>(X + p * N1X * XPITCH, q, dA, dA + P);
    }
    __syncthreads();
  }
  cplx<T> *dst = S + (size_t)j * NZ * P;
  for (int c0 = 0; c0 < P; c0 += CW) {
    const int nc = min(CW, P - c0);
    for (int job = tid; job < CW * N1Z; job += kPlaneThreads_) {
      const int n1 = job / CW, c = job - n1 * CW;
      if (c < nc)
        col_step1<T, NZ, false, CW>(plane + c0 + c, P, n1, tw2z, X + n1 * N2Z * CW + c, false, mk<T>((T)0, (T)0));
    }
    __syncthreads();
    for (int job = tid; job < CW * N2Z; job += kPlaneThreads_) {
      const int k2 = job / CW, c = job - k2 * CW;
      if (c < nc) {
        const cplx<T> u0 = col_step3<T, NZ, false, CW>(X, c, k2, dst + c0 + c, P);
        if (zrhs && c0 + c == 0 && k2 == 0) zrhs[j] = (double)u0.x;
      }
    }
    __syncthreads();
  }
}

// Inverse: spectrum plane -> out = addend + scale * result.
template <typename T, int NX, int NZ>
__global__ void __launch_bounds__(PlaneCfg<T, NX, NZ>::THREADS)
k_plane_inv(Ptr3<cplx<T> *> S_, Ptr3<T *> out_, Ptr3<const T *> add_, const cplx<T> *__restrict__ twx,
            const cplx<T> *__restrict__ twz, T scale, const double *zsol) {
  const cplx<T> *__restrict__ S = S_[blockIdx.y];
  T *out = out_[blockIdx.y];
  const T *addend = add_[blockIdx.y];
  using Cfg = PlaneCfg<T, NX, NZ>;
  constexpr int P = Cfg::P, N1X = Cfg::N1X, N2X = Cfg::N2X, XPITCH = Cfg::XPITCH, CP = Cfg::CP, CW = Cfg::CW;
  constexpr int kPlaneThreads_ = Cfg::THREADS;
  constexpr int N1Z = TwoStep<NZ>::N1, N2Z = TwoStep<NZ>::N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *tw2x = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *tw2z = tw2x + NX;
  cplx<T> *plane = tw2z + NZ;
  cplx<T> *X = plane + NZ * P;
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  load_step_twiddles<T, NX>(tw2x, twx);
  load_step_twiddles<T, NZ>(tw2z, twz);
  pdl_wait();  // the fields below are the predecessor's output
  __syncthreads();
  const cplx<T> *src = S + (size_t)j * NZ * P;
  const cplx<T> z0 = zsol ? mk<T>((T)zsol[j], (T)0) : mk<T>((T)0, (T)0);
  for (int c0 = 0; c0 < P; c0 += CW) {
    const int nc = min(CW, P - c0);
    for (int job = tid; job < CW * N1Z; job += kPlaneThreads_) {
      const int n1 = job / CW, c = job - n1 * CW;
      if (c < nc)
        col_step1<T, NZ, true, CW>(src + c0 + c, P, n1, tw2z, X + n1 * N2Z * CW + c, zsol && c0 + c == 0, z0);
    }
    __syncthreads();
    for (int job = tid; job < CW * N2Z; job += kPlaneThreads_) {
      const int k2 = job / CW, c = job - k2 * CW;
      if (c < nc) col_step3<T, NZ, true, CW>(X, c, k2, plane + c0 + c, P);
    }
    __syncthreads();
  }
  T *dst = out + (size_t)j * NZ * NX;
  const T *add = addend ? addend + (size_t)j * NZ * NX : nullptr;
  for (int p0 = 0; p0 < NZ / 2; p0 += CP) {
    const int np = min(CP, NZ / 2 - p0);
    for (int job = tid; job < np * N1X; job += kPlaneThreads_) {
      const int p = job / N1X, n1 = job - p * N1X;
      const cplx<T> *sA = plane + (p0 + p) * 2 * P;
      rinv_step1<T, NX>(sA, sA + P, n1, tw2x, X + (p * N1X + n1) * XPITCH);
    }
    __syncthreads();
    for (int job = tid; job < np * N2X; job += kPlaneThreads_) {
      const int p = job / N2X, k2 = job - p * N2X;
      const size_t r = (size_t)(p0 + p) * 2 * NX;
      rinv_step3<T, NX, XPITCH>(X + p * N1X * XPITCH, k2, dst + r, dst + r + NX, add ? add + r : nullptr,
                                add ? add + r + NX : nullptr, scale);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
#define IBM_FOR_EACH_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

// plane kernels are instantiated for square-ish planes whose spectrum fits in shared memory
#define IBM_PLANE_SHAPES(X)                                                    \
  X(8, 8) X(12, 12) X(16, 16) X(24, 24) X(32, 32) X(48, 48) X(64, 64) X(96, 96) \
  X(128, 128) X(192, 192) X(256, 128) X(128, 256) X(64, 128) X(128, 64)

template <typename T> static bool plane_supported(int nx, int nz) {
#define X(a, b) if (nx == a && nz == b) return PlaneCfg<T, a, b>::ok;
  IBM_PLANE_SHAPES(X)
#undef X
  return false;
}

template <typename T>
cudaError_t launch_forward(const TransformGeom &g, Ptr3<const T *> in, Ptr3<cplx<T> *> S, const cplx<T> *twx,
                           const cplx<T> *twz, T in_scale, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if constexpr (sizeof(T) == 4) {
    if (g.use_plane == kPlaneDft && g.dft_fwd) return launch_dft_forward(g, in, S, in_scale, st);
  }
  if (g.use_plane >= 2 && cplane_supported<T>(nx, nz, g.use_plane))
    return launch_cplane_forward<T>(g, g.use_plane, in, S, twx, twz, in_scale, st);
  if (g.use_plane == 1 && plane_supported<T>(nx, nz)) {
#define X(a, b)                                                                                  \
  if (nx == a && nz == b) {                                                                      \
    if constexpr (PlaneCfg<T, a, b>::ok) {                                                       \
      { cudaError_t e = ensure_max_smem<k_plane_fwd<T, a, b>>(); if (e) return e; }              \
      IBM_KTRY(launch_pdl(k_plane_fwd<T, a, b>, dim3(ny, g.nb), PlaneCfg<T, a, b>::THREADS, PlaneCfg<T, a, b>::bytes, st, in, S, twx, twz, in_scale, g.zrhs)); \
      return cudaGetLastError();                                                                 \
    }                                                                                            \
  }
    IBM_PLANE_SHAPES(X)
#undef X
  }
  // axis path: x rows then z columns
  return launch_axis_forward<T>(g, in, S, twx, twz, in_scale, st);
}

template <typename T>
cudaError_t launch_inverse(const TransformGeom &g, Ptr3<cplx<T> *> S, Ptr3<T *> out, Ptr3<const T *> addend,
                           const cplx<T> *twx, const cplx<T> *twz, T scale, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if constexpr (sizeof(T) == 4) {
    if (g.use_plane == kPlaneDft && g.dft_inv) return launch_dft_inverse(g, S, out, addend, scale, st);
  }
  if (g.use_plane >= 2 && cplane_supported<T>(nx, nz, g.use_plane))
    return launch_cplane_inverse<T>(g, g.use_plane, S, out, addend, twx, twz, scale, st);
  if (g.use_plane == 1 && plane_supported<T>(nx, nz)) {
#define X(a, b)                                                                                  \
  if (nx == a && nz == b) {                                                                      \
    if constexpr (PlaneCfg<T, a, b>::ok) {                                                       \
      { cudaError_t e = ensure_max_smem<k_plane_inv<T, a, b>>(); if (e) return e; }              \
      IBM_KTRY(launch_pdl(k_plane_inv<T, a, b>, dim3(ny, g.nb), PlaneCfg<T, a, b>::THREADS, PlaneCfg<T, a, b>::bytes, st, S, out, addend, twx, twz, scale, g.zsol)); \
      return cudaGetLastError();                                                                 \
    }                                                                                            \
  }
    IBM_PLANE_SHAPES(X)
#undef X
  }
  return launch_axis_inverse<T>(g, S, out, addend, twx, twz, scale, st);
}

template cudaError_t launch_forward<float>(const TransformGeom &, Ptr3<const float *>, Ptr3<float2 *>, const float2 *,
                                           const float2 *, float, cudaStream_t);
template cudaError_t launch_forward<double>(const TransformGeom &, Ptr3<const double *>, Ptr3<double2 *>,
                                            const double2 *, const double2 *, double, cudaStream_t);
template cudaError_t launch_inverse<float>(const TransformGeom &, Ptr3<float2 *>, Ptr3<float *>, Ptr3<const float *>,
                                           const float2 *, const float2 *, float, cudaStream_t);
template cudaError_t launch_inverse<double>(const TransformGeom &, Ptr3<double2 *>, Ptr3<double *>,
                                            Ptr3<const double *>, const double2 *, const double2 *, double,
                                            cudaStream_t);

template <typename T> int transform_launches(const TransformGeom &g) {
  if (g.use_plane == kPlaneDft) return (sizeof(T) == 4 && g.dft_fwd) ? 1 : 2;
  if (g.use_plane >= 2) return cplane_supported<T>(g.nx, g.nz, g.use_plane) ? 1 : 2;
  return (g.use_plane == 1 && plane_supported<T>(g.nx, g.nz)) ? 1 : 2;
}
template int transform_launches<float>(const TransformGeom &);
template int transform_launches<double>(const TransformGeom &);

template <typename T> int plane_modes(int nx, int nz, int *modes) {
  int n = 0;
  if (sizeof(T) == 4 && dft_tc_supported(nx, nz)) modes[n++] = kPlaneDft;
  modes[n++] = 0;
  if (plane_supported<T>(nx, nz)) modes[n++] = 1;
  for (int c = 2; c <= 8; c *= 2)
    if (cplane_supported<T>(nx, nz, c)) modes[n++] = c;
  return n;
}
template int plane_modes<float>(int, int, int *);
template int plane_modes<double>(int, int, int *);

template <typename T> int default_plane_mode(int nx, int ny, int nz) {
  // Measured on GB300 (128^3 to 384x256x256): in FP32 the one-CTA plane
  // kernels win up to 128 x 256 planes and the split passes from 192^2 on;
  // in FP64 (arithmetic-bound here) the split passes win at every size.
  // The cluster kernels lose to both and stay available to the tuner and to
  // IBM_PLANE_MODE.
  (void)ny;
  if (sizeof(T) == 4 && plane_supported<T>(nx, nz) && nx * nz <= 128 * 256) return 1;
  return 0;
}
template int default_plane_mode<float>(int, int, int);
template int default_plane_mode<double>(int, int, int);

bool transform_size_supported(int n) {
#define X(N) if (n == N) return true;
  IBM_FOR_EACH_N(X)
#undef X
  return false;
}

}  // namespace ibm
