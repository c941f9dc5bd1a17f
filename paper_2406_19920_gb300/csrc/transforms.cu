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
// Two kernel families:
//   plane kernels  one CTA per y-plane, the whole plane staged in shared
//                  memory: x-FFT of every row pair, then z-FFT of every
//                  column, then one coalesced store (one HBM read + one write
//                  per direction);
//   axis kernels   for planes larger than shared memory: x-rows and
//                  z-columns in separate passes.
#include "fft.cuh"
#include "internal.h"
#include "tma.cuh"

namespace ibm {

constexpr int kThreads = 256;

// --------------------------------------------------------------------------
// plane kernels: one CTA per y-plane, the plane moved by bulk async copies
// --------------------------------------------------------------------------
constexpr int kPlaneThreads = 512;

// shared-memory layout of a plane kernel (bytes from the dynamic base):
//   [0, 16)            mbarrier
//   staging            NZ*NX reals (forward input / inverse addend)
//   twx, twz           NX + NZ complex twiddles
//   plane              NZ rows of P = NX/2+1 complex (NZ/2 pairs of NX+2)
template <typename T, int NX, int NZ> struct PlaneLayout {
  static constexpr int P = NX / 2 + 1;
  static constexpr size_t staging = 16;
  static constexpr size_t tw = staging + sizeof(T) * (size_t)NZ * NX;
  static constexpr size_t plane = tw + sizeof(cplx<T>) * (size_t)(NX + NZ);
  static constexpr size_t bytes = plane + sizeof(cplx<T>) * (size_t)NZ * P;
  static_assert(tw % 16 == 0 && plane % 16 == 0, "16-byte aligned regions");
};

template <typename T, int NX, int NZ>
__global__ void __launch_bounds__(kPlaneThreads)
k_plane_fwd(const T *__restrict__ in, cplx<T> *__restrict__ S, const cplx<T> *__restrict__ twx_g,
            const cplx<T> *__restrict__ twz_g, T in_scale, int *err, double *zrhs) {
  using L = PlaneLayout<T, NX, NZ>;
  constexpr int P = L::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  T *real = reinterpret_cast<T *>(smem_raw + L::staging);
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw + L::tw);
  cplx<T> *twz = twx + NX;
  cplx<T> *plane = reinterpret_cast<cplx<T> *>(smem_raw + L::plane);
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  constexpr uint32_t kInBytes = sizeof(T) * NZ * NX;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, kInBytes);
    bulk_g2s(real, in + (size_t)j * NZ * NX, kInBytes, bar);
  }
  load_twiddles<T>(twx, twx_g, NX);
  load_twiddles<T>(twz, twz_g, NZ);
  if (!__syncthreads_and(mbar_wait(bar, 0, err))) return;
  {  // x: complex FFT of each row pair z = a + i b, then split into two half spectra
    constexpr int G = FftPlan<NX>::G;
    constexpr int NG = kPlaneThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < NZ / 2; base += NG) {
      const int p = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, p < NZ / 2);
      if (p >= NZ / 2) continue;
      cplx<T> *row = plane + p * (NX + 2);
      const T *ra = real + (2 * p) * NX;
      for (int n = lg; n < NX; n += G) row[n] = mk<T>(ra[n] * in_scale, ra[NX + n] * in_scale);
      __syncwarp(mask);
      fft_row<T, NX, false>(row, 1, twx, lg, mask);
      split_pair<T, NX>(row, row, row + P, 1, lg, mask);
    }
  }
  __syncthreads();
  {  // z: complex FFT of each of the P columns (stride P)
    constexpr int G = FftPlan<NZ>::G;
    constexpr int NG = kPlaneThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < P; base += NG) {
      const int c = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, c < P);
      if (c >= P) continue;
      fft_row<T, NZ, false>(plane + c, P, twz, lg, mask);
    }
  }
  fence_proxy_async();
  __syncthreads();
  if (tid == 0) {
    if (zrhs) zrhs[j] = (double)plane[0].x;
    bulk_s2g(S + (size_t)j * NZ * P, plane, (uint32_t)(sizeof(cplx<T>) * NZ * P));
    bulk_commit();
    bulk_wait_read();
  }
}

// Inverse: spectrum plane -> real plane, out = addend + scale * result.
template <typename T, int NX, int NZ>
__global__ void __launch_bounds__(kPlaneThreads)
k_plane_inv(const cplx<T> *__restrict__ S, T *out, const T *addend, const cplx<T> *__restrict__ twx_g,
            const cplx<T> *__restrict__ twz_g, T scale, int *err, const double *zsol) {
  using L = PlaneLayout<T, NX, NZ>;
  constexpr int P = L::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  T *addb = reinterpret_cast<T *>(smem_raw + L::staging);
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw + L::tw);
  cplx<T> *twz = twx + NX;
  cplx<T> *plane = reinterpret_cast<cplx<T> *>(smem_raw + L::plane);
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  constexpr uint32_t kSpecBytes = sizeof(cplx<T>) * NZ * P;
  constexpr uint32_t kAddBytes = sizeof(T) * NZ * NX;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, kSpecBytes + (addend ? kAddBytes : 0u));
    bulk_g2s(plane, S + (size_t)j * NZ * P, kSpecBytes, bar);
    if (addend) bulk_g2s(addb, addend + (size_t)j * NZ * NX, kAddBytes, bar);
  }
  load_twiddles<T>(twx, twx_g, NX);
  load_twiddles<T>(twz, twz_g, NZ);
  if (!__syncthreads_and(mbar_wait(bar, 0, err))) return;
  if (zsol) {
    if (tid == 0) plane[0] = mk<T>((T)zsol[j], (T)0);
    __syncthreads();
  }
  {
    constexpr int G = FftPlan<NZ>::G;
    constexpr int NG = kPlaneThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < P; base += NG) {
      const int c = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, c < P);
      if (c >= P) continue;
      fft_row<T, NZ, true>(plane + c, P, twz, lg, mask);
    }
  }
  __syncthreads();
  {
    constexpr int G = FftPlan<NX>::G;
    constexpr int NG = kPlaneThreads / G;
    const int gid = tid / G, lg = tid % G;
    T *dst = out + (size_t)j * NZ * NX;
    for (int base = 0; base < NZ / 2; base += NG) {
      const int p = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, p < NZ / 2);
      if (p >= NZ / 2) continue;
      cplx<T> *row = plane + p * (NX + 2);
      merge_pair<T, NX>(row, row + P, 1, row, lg, mask);
      fft_row<T, NX, true>(row, 1, twx, lg, mask);
      T *d0 = dst + (size_t)(2 * p) * NX;
      const T *a0 = addb + (2 * p) * NX;
      for (int n = lg; n < NX; n += G) {
        const cplx<T> z = row[n];
        T v0 = z.x * scale, v1 = z.y * scale;
        if (addend) { v0 += a0[n]; v1 += a0[NX + n]; }
        d0[n] = v0;
        d0[NX + n] = v1;
      }
    }
  }
}

// --------------------------------------------------------------------------
// axis kernels (planes larger than shared memory)
// --------------------------------------------------------------------------

// x forward: a CTA takes PPC row pairs of one plane.  grid (ceil(NZ/2/PPC), ny)
template <typename T, int NX>
__global__ void __launch_bounds__(kThreads)
k_xfwd_rows(const T *__restrict__ in, cplx<T> *__restrict__ S, const cplx<T> *__restrict__ twx_g, int nz,
            T in_scale) {
  constexpr int P = NX / 2 + 1;
  constexpr int G = FftPlan<NX>::G;
  constexpr int PPC = kThreads / G;  // pairs per CTA
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *buf = twx + NX;  // PPC rows of NX
  const int j = blockIdx.y;
  const int p0 = blockIdx.x * PPC;
  const int np = min(PPC, nz / 2 - p0);
  const int tid = threadIdx.x;
  load_twiddles<T>(twx, twx_g, NX);
  {
    const T *src = in + ((size_t)j * nz + 2 * p0) * NX;
    T *bf = reinterpret_cast<T *>(buf);
    for (int idx = tid; idx < np * 2 * NX; idx += kThreads) {
      const int k = idx / NX, n = idx - k * NX;
      bf[((k >> 1) * NX + n) * 2 + (k & 1)] = src[idx] * in_scale;
    }
  }
  __syncthreads();
  const int gid = tid / G, lg = tid % G;
  const unsigned mask = __ballot_sync(0xffffffffu, gid < np);
  if (gid >= np) return;
  cplx<T> *row = buf + gid * NX;
  fft_row<T, NX, false>(row, 1, twx, lg, mask);
  cplx<T> *dA = S + ((size_t)j * nz + 2 * (p0 + gid)) * P;
  split_pair<T, NX>(row, dA, dA + P, 1, lg, mask);
}

// x inverse.  out = addend + scale * result
template <typename T, int NX>
__global__ void __launch_bounds__(kThreads)
k_xinv_rows(const cplx<T> *__restrict__ S, T *out, const T *addend, const cplx<T> *__restrict__ twx_g,
            int nz, T scale) {
  constexpr int P = NX / 2 + 1;
  constexpr int G = FftPlan<NX>::G;
  constexpr int PPC = kThreads / G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *buf = twx + NX;
  const int j = blockIdx.y;
  const int p0 = blockIdx.x * PPC;
  const int np = min(PPC, nz / 2 - p0);
  const int tid = threadIdx.x;
  load_twiddles<T>(twx, twx_g, NX);
  __syncthreads();
  const int gid = tid / G, lg = tid % G;
  const unsigned mask = __ballot_sync(0xffffffffu, gid < np);
  if (gid >= np) return;
  const int p = p0 + gid;
  cplx<T> *row = buf + gid * NX;
  const cplx<T> *sA = S + ((size_t)j * nz + 2 * p) * P;
  merge_pair<T, NX>(sA, sA + P, 1, row, lg, mask);
  fft_row<T, NX, true>(row, 1, twx, lg, mask);
  T *d0 = out + ((size_t)j * nz + 2 * p) * NX;
  const T *a0 = addend ? addend + ((size_t)j * nz + 2 * p) * NX : nullptr;
  for (int n = lg; n < NX; n += G) {
    const cplx<T> z = row[n];
    T v0 = z.x * scale, v1 = z.y * scale;
    if (a0) { v0 += a0[n]; v1 += a0[NX + n]; }
    d0[n] = v0;
    d0[NX + n] = v1;
  }
}

// z columns, in place: a CTA takes W consecutive kx columns of one plane.
// grid (ceil(P / W), ny), block W * G lanes.
template <typename T, int NZ, bool INV, int W>
__global__ void __launch_bounds__(1024)
k_zcols(cplx<T> *__restrict__ S, const cplx<T> *__restrict__ twz_g, int P, double *zrhs, const double *zsol) {
  constexpr int G = FftPlan<NZ>::G;
  constexpr int PITCH = W + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T> *twz = reinterpret_cast<cplx<T> *>(smem_raw);
  cplx<T> *tile = twz + NZ;  // [NZ][PITCH]
  const int j = blockIdx.y;
  const int c0 = blockIdx.x * W;
  const int nc = min(W, P - c0);
  const int tid = threadIdx.x;
  const int nthr = W * G;
  load_twiddles<T>(twz, twz_g, NZ);
  cplx<T> *base = S + (size_t)j * NZ * P + c0;
  for (int idx = tid; idx < NZ * W; idx += nthr) {
    const int k = idx / W, c = idx - k * W;
    if (c < nc) tile[k * PITCH + c] = base[(size_t)k * P + c];
  }
  __syncthreads();
  if (INV && zsol && c0 == 0 && tid == 0) tile[0] = mk<T>((T)zsol[j], (T)0);
  __syncthreads();
  {
    const int gid = tid / G, lg = tid % G;
    const unsigned mask = __ballot_sync(warp_full_mask(), gid < nc);
    if (gid < nc) fft_row<T, NZ, INV>(tile + gid, PITCH, twz, lg, mask);
  }
  __syncthreads();
  if (!INV && zrhs && c0 == 0 && tid == 0) zrhs[j] = (double)tile[0].x;
  for (int idx = tid; idx < NZ * W; idx += nthr) {
    const int k = idx / W, c = idx - k * W;
    if (c < nc) base[(size_t)k * P + c] = tile[k * PITCH + c];
  }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
template <typename T> size_t plane_smem_bytes(int nx, int nz) {
  return 16 + sizeof(T) * (size_t)nz * nx + sizeof(cplx<T>) * ((size_t)nx + nz + (size_t)nz * (nx / 2 + 1));
}

template <typename T> constexpr int zcols_width() { return sizeof(T) == 4 ? 16 : 8; }

#define IBM_FOR_EACH_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

// plane kernels are instantiated for square-ish planes that fit in shared memory
#define IBM_PLANE_SHAPES(X)                                                    \
  X(8, 8) X(12, 12) X(16, 16) X(24, 24) X(32, 32) X(48, 48) X(64, 64) X(96, 96) \
  X(128, 128) X(192, 192) X(256, 128) X(128, 256) X(64, 128) X(128, 64)

template <typename T> static bool plane_supported(int nx, int nz) {
#define X(a, b) if (nx == a && nz == b) return plane_smem_bytes<T>(nx, nz) <= kPlaneSmemLimit;
  IBM_PLANE_SHAPES(X)
#undef X
  return false;
}

template <typename T>
cudaError_t launch_forward(const TransformGeom &g, const T *in, cplx<T> *S, const cplx<T> *twx,
                           const cplx<T> *twz, T in_scale, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, P = nx / 2 + 1;
  if (g.use_plane >= 2 && cplane_supported<T>(nx, nz, g.use_plane))
    return launch_cplane_forward<T>(g, g.use_plane, in, S, twx, twz, in_scale, st);
  if (g.use_plane == 1 && plane_supported<T>(nx, nz)) {
    const size_t bytes = plane_smem_bytes<T>(nx, nz);
#define X(a, b)                                                                     \
  if (nx == a && nz == b) {                                                         \
    if (plane_smem_bytes<T>(a, b) <= kPlaneSmemLimit) {                             \
      { cudaError_t e = ensure_max_smem<k_plane_fwd<T, a, b>>(); if (e) return e; } \
      k_plane_fwd<T, a, b><<<ny, kPlaneThreads, bytes, st>>>(in, S, twx, twz, in_scale, g.err, g.zrhs);  \
      return cudaGetLastError();                                                    \
    }                                                                               \
  }
    IBM_PLANE_SHAPES(X)
#undef X
  }
  // axis path: x rows then z columns
  bool done = false;
#define X(N)                                                                               \
  if (nx == N) {                                                                           \
    constexpr int PPC = kThreads / FftPlan<N>::G;                                          \
    const size_t bytes = sizeof(cplx<T>) * ((size_t)N + (size_t)PPC * N);                 \
    dim3 grid(ceil_div(nz / 2, PPC), ny);                                                  \
    { cudaError_t e = ensure_max_smem<k_xfwd_rows<T, N>>(); if (e) return e; }                    \
    k_xfwd_rows<T, N><<<grid, kThreads, bytes, st>>>(in, S, twx, nz, in_scale);            \
    done = true;                                                                           \
  }
  IBM_FOR_EACH_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  done = false;
  constexpr int W = zcols_width<T>();
#define X(N)                                                                               \
  if (nz == N) {                                                                           \
    const size_t bytes = sizeof(cplx<T>) * ((size_t)N + (size_t)N * (W + 1));              \
    { cudaError_t e = ensure_max_smem<k_zcols<T, N, false, W>>(); if (e) return e; }                    \
    dim3 grid(ceil_div(P, W), ny);                                                         \
    k_zcols<T, N, false, W><<<grid, W * FftPlan<N>::G, bytes, st>>>(S, twz, P, g.zrhs, nullptr);            \
    done = true;                                                                           \
  }
  IBM_FOR_EACH_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inverse(const TransformGeom &g, cplx<T> *S, T *out, const T *addend, const cplx<T> *twx,
                           const cplx<T> *twz, T scale, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, P = nx / 2 + 1;
  if (g.use_plane >= 2 && cplane_supported<T>(nx, nz, g.use_plane))
    return launch_cplane_inverse<T>(g, g.use_plane, S, out, addend, twx, twz, scale, st);
  if (g.use_plane == 1 && plane_supported<T>(nx, nz)) {
    const size_t bytes = plane_smem_bytes<T>(nx, nz);
#define X(a, b)                                                                     \
  if (nx == a && nz == b) {                                                         \
    if (plane_smem_bytes<T>(a, b) <= kPlaneSmemLimit) {                             \
      { cudaError_t e = ensure_max_smem<k_plane_inv<T, a, b>>(); if (e) return e; } \
      k_plane_inv<T, a, b><<<ny, kPlaneThreads, bytes, st>>>(S, out, addend, twx, twz, scale, g.err, g.zsol); \
      return cudaGetLastError();                                                    \
    }                                                                               \
  }
    IBM_PLANE_SHAPES(X)
#undef X
  }
  bool done = false;
  constexpr int W = zcols_width<T>();
#define X(N)                                                                               \
  if (nz == N) {                                                                           \
    const size_t bytes = sizeof(cplx<T>) * ((size_t)N + (size_t)N * (W + 1));              \
    { cudaError_t e = ensure_max_smem<k_zcols<T, N, true, W>>(); if (e) return e; }                    \
    dim3 grid(ceil_div(P, W), ny);                                                         \
    k_zcols<T, N, true, W><<<grid, W * FftPlan<N>::G, bytes, st>>>(S, twz, P, nullptr, g.zsol);             \
    done = true;                                                                           \
  }
  IBM_FOR_EACH_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  done = false;
#define X(N)                                                                               \
  if (nx == N) {                                                                           \
    constexpr int PPC = kThreads / FftPlan<N>::G;                                          \
    const size_t bytes = sizeof(cplx<T>) * ((size_t)N + (size_t)PPC * N);                 \
    dim3 grid(ceil_div(nz / 2, PPC), ny);                                                  \
    { cudaError_t e = ensure_max_smem<k_xinv_rows<T, N>>(); if (e) return e; }                    \
    k_xinv_rows<T, N><<<grid, kThreads, bytes, st>>>(S, out, addend, twx, nz, scale);       \
    done = true;                                                                           \
  }
  IBM_FOR_EACH_N(X)
#undef X
  if (!done) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template cudaError_t launch_forward<float>(const TransformGeom &, const float *, float2 *, const float2 *,
                                           const float2 *, float, cudaStream_t);
template cudaError_t launch_forward<double>(const TransformGeom &, const double *, double2 *, const double2 *,
                                            const double2 *, double, cudaStream_t);
template cudaError_t launch_inverse<float>(const TransformGeom &, float2 *, float *, const float *,
                                           const float2 *, const float2 *, float, cudaStream_t);
template cudaError_t launch_inverse<double>(const TransformGeom &, double2 *, double *, const double *,
                                            const double2 *, const double2 *, double, cudaStream_t);

template <typename T> int transform_launches(const TransformGeom &g) {
  if (g.use_plane >= 2) return cplane_supported<T>(g.nx, g.nz, g.use_plane) ? 1 : 2;
  return (g.use_plane == 1 && plane_supported<T>(g.nx, g.nz)) ? 1 : 2;
}
template int transform_launches<float>(const TransformGeom &);
template int transform_launches<double>(const TransformGeom &);

template <typename T> int plane_modes(int nx, int nz, int *modes) {
  int n = 0;
  modes[n++] = 0;
  if (plane_supported<T>(nx, nz)) modes[n++] = 1;
  for (int c = 2; c <= 8; c *= 2)
    if (cplane_supported<T>(nx, nz, c)) modes[n++] = c;
  return n;
}
template int plane_modes<float>(int, int, int *);
template int plane_modes<double>(int, int, int *);

template <typename T> int default_plane_mode(int nx, int ny, int nz) {
  // Measured on GB300 (FP32 and FP64, 128^3 to 384x256x256): the one-CTA
  // plane kernels beat the split passes where they fit, and the cluster
  // kernels lose to both (their row/column exchange through distributed
  // shared memory costs more than the L2 round trip of the split passes).
  // Clusters stay available to the tuner and to IBM_PLANE_MODE.
  (void)ny;
  return plane_supported<T>(nx, nz) ? 1 : 0;
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
