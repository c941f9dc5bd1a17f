// cplane.cu -- plane transforms by a thread-block cluster of C CTAs per y-plane.
//
// Same transform as the one-CTA plane kernels (real FFT along x of row pairs
// packed as z = a + i b, complex FFT along z), for planes that do not fit
// one CTA's shared memory or that leave SMs idle with one CTA per plane:
//   forward  CTA r of the cluster bulk-loads z-rows [r R, (r+1) R) (R = NZ/C),
//            x-transforms them into its row buffer; cluster barrier; gathers
//            kx columns [r Pc, (r+1) Pc) of all NZ rows from the row buffers
//            of the whole cluster through distributed shared memory; cluster
//            barrier; z-transforms its columns and stores them;
//   inverse  the mirror: columns loaded and z-inverted, cluster barrier,
//            rows gathered through distributed shared memory, cluster
//            barrier, c2r per row pair, the addend read alongside the stores.
// Every CTA reaches every cluster barrier (a failed bounded wait only
// suppresses the stores), so no barrier can be left waiting.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "internal.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace ibm {

constexpr int kCThreads = 256;

// Shared memory of one CTA (bytes from the dynamic base):
//   [0, 16)  mbarrier (forward)
//   tw       NX + NZ complex twiddles
//   xbuf     R z-rows of P = NX/2+1 complex (R/2 pairs of NX+2): x-transformed rows
//   zbuf     NZ rows of PCP complex: this CTA's kx columns
//   stage    R*NX reals: forward input, aliasing zbuf (dead before zbuf is filled)
template <typename T, int NX, int NZ, int C> struct CLayout {
  static constexpr int P = NX / 2 + 1;
  static constexpr int R = NZ / C;                    // z-rows per CTA
  static constexpr int PC = (P + C - 1) / C;          // kx columns per CTA
  static constexpr int PCP = (PC % 2) ? PC : PC + 1;  // odd pitch: column FFTs spread over banks
  static constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr size_t tw = 16;
  static constexpr size_t xbuf = tw + align16(sizeof(cplx<T>) * (size_t)(NX + NZ));
  static constexpr size_t zbuf = xbuf + align16(sizeof(cplx<T>) * (size_t)R * P);
  static constexpr size_t zbytes = align16(sizeof(cplx<T>) * (size_t)NZ * PCP);
  static constexpr size_t sbytes = align16(sizeof(T) * (size_t)R * NX);
  static constexpr size_t fwd_stage = zbuf;
  static constexpr size_t fwd_bytes = zbuf + (zbytes > sbytes ? zbytes : sbytes);
  static constexpr size_t inv_bytes = zbuf + zbytes;  // <= fwd_bytes
  static_assert(NZ % C == 0 && R % 2 == 0, "a CTA owns whole row pairs");
  static_assert(P <= C * PC, "columns cover the half spectrum");
};

template <typename T, int NX, int NZ, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kCThreads)
k_cplane_fwd(Ptr3<const T *> in_, Ptr3<cplx<T> *> S_, const cplx<T> *__restrict__ twx_g,
             const cplx<T> *__restrict__ twz_g, T in_scale, int *err, double *zrhs) {
  pdl_wait();
  const T *__restrict__ in = in_[blockIdx.y];
  cplx<T> *__restrict__ S = S_[blockIdx.y];
  using L = CLayout<T, NX, NZ, C>;
  constexpr int P = L::P, R = L::R, PC = L::PC, PCP = L::PCP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int j = blockIdx.x / C;
  const int tid = threadIdx.x;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  T *stage = reinterpret_cast<T *>(smem_raw + L::fwd_stage);  // dead once the rows are transformed
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw + L::tw);
  cplx<T> *twz = twx + NX;
  cplx<T> *xbuf = reinterpret_cast<cplx<T> *>(smem_raw + L::xbuf);
  cplx<T> *zbuf = reinterpret_cast<cplx<T> *>(smem_raw + L::zbuf);
  constexpr uint32_t kInBytes = sizeof(T) * R * NX;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, kInBytes);
    bulk_g2s(stage, in + ((size_t)j * NZ + (size_t)r * R) * NX, kInBytes, bar);
  }
  load_twiddles<T>(twx, twx_g, NX);
  load_twiddles<T>(twz, twz_g, NZ);
  const bool ok = __syncthreads_and(mbar_wait(bar, 0, err));
  {  // x: row pairs of this CTA
    constexpr int G = FftPlan<NX>::G;
    constexpr int NG = kCThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < R / 2; base += NG) {
      const int p = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, p < R / 2);
      if (p >= R / 2) continue;
      cplx<T> *row = xbuf + p * (NX + 2);
      const T *ra = stage + (2 * p) * NX;
      for (int n = lg; n < NX; n += G) row[n] = mk<T>(ra[n] * in_scale, ra[NX + n] * in_scale);
      __syncwarp(mask);
      fft_row<T, NX, false>(row, 1, twx, lg, mask);
      split_pair<T, NX>(row, row, row + P, 1, lg, mask);
    }
  }
  cluster.sync();
  // gather kx columns [c0, c0 + nc) of all NZ rows from the cluster's row buffers
  const int c0 = r * PC;
  const int nc = min(PC, P - c0);
  for (int idx = tid; idx < NZ * PC; idx += kCThreads) {
    const int kz = idx / PC, c = idx - kz * PC;
    if (c < nc) {
      const cplx<T> *src = cluster.map_shared_rank(xbuf, kz / R);
      zbuf[kz * PCP + c] = src[(kz % R) * P + c0 + c];
    }
  }
  cluster.sync();
  {  // z: columns of this CTA
    constexpr int G = FftPlan<NZ>::G;
    constexpr int NG = kCThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < nc; base += NG) {
      const int c = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, c < nc);
      if (c >= nc) continue;
      fft_row<T, NZ, false>(zbuf + c, PCP, twz, lg, mask);
    }
  }
  __syncthreads();
  if (!ok) return;
  if (zrhs && r == 0 && tid == 0) zrhs[j] = (double)zbuf[0].x;
  cplx<T> *dst = S + (size_t)j * NZ * P + c0;
  for (int idx = tid; idx < NZ * PC; idx += kCThreads) {
    const int kz = idx / PC, c = idx - kz * PC;
    if (c < nc) dst[(size_t)kz * P + c] = zbuf[kz * PCP + c];
  }
}

template <typename T, int NX, int NZ, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kCThreads)
k_cplane_inv(Ptr3<cplx<T> *> S_, Ptr3<T *> out_, Ptr3<const T *> add_, const cplx<T> *__restrict__ twx_g,
             const cplx<T> *__restrict__ twz_g, T scale, int *err, const double *zsol) {
  pdl_wait();
  const cplx<T> *__restrict__ S = S_[blockIdx.y];
  T *out = out_[blockIdx.y];
  const T *addend = add_[blockIdx.y];
  using L = CLayout<T, NX, NZ, C>;
  constexpr int P = L::P, R = L::R, PC = L::PC, PCP = L::PCP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int j = blockIdx.x / C;
  const int tid = threadIdx.x;
  cplx<T> *twx = reinterpret_cast<cplx<T> *>(smem_raw + L::tw);
  cplx<T> *twz = twx + NX;
  cplx<T> *xbuf = reinterpret_cast<cplx<T> *>(smem_raw + L::xbuf);
  cplx<T> *zbuf = reinterpret_cast<cplx<T> *>(smem_raw + L::zbuf);
  load_twiddles<T>(twx, twx_g, NX);
  load_twiddles<T>(twz, twz_g, NZ);
  const int c0 = r * PC;
  const int nc = min(PC, P - c0);
  {  // this CTA's kx columns of the spectrum plane
    const cplx<T> *src = S + (size_t)j * NZ * P + c0;
    for (int idx = tid; idx < NZ * PC; idx += kCThreads) {
      const int kz = idx / PC, c = idx - kz * PC;
      if (c < nc) zbuf[kz * PCP + c] = src[(size_t)kz * P + c];
    }
  }
  __syncthreads();
  if (zsol && r == 0 && tid == 0) zbuf[0] = mk<T>((T)zsol[j], (T)0);
  __syncthreads();
  {
    constexpr int G = FftPlan<NZ>::G;
    constexpr int NG = kCThreads / G;
    const int gid = tid / G, lg = tid % G;
    for (int base = 0; base < nc; base += NG) {
      const int c = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, c < nc);
      if (c >= nc) continue;
      fft_row<T, NZ, true>(zbuf + c, PCP, twz, lg, mask);
    }
  }
  cluster.sync();
  // gather the full kx range of this CTA's z-rows
  for (int idx = tid; idx < R * P; idx += kCThreads) {
    const int lr = idx / P, kx = idx - lr * P;
    const cplx<T> *src = cluster.map_shared_rank(zbuf, kx / PC);
    xbuf[idx] = src[(r * R + lr) * PCP + (kx % PC)];
  }
  cluster.sync();
  {
    constexpr int G = FftPlan<NX>::G;
    constexpr int NG = kCThreads / G;
    const int gid = tid / G, lg = tid % G;
    T *dst = out + ((size_t)j * NZ + (size_t)r * R) * NX;
    for (int base = 0; base < R / 2; base += NG) {
      const int p = base + gid;
      const unsigned mask = __ballot_sync(0xffffffffu, p < R / 2);
      if (p >= R / 2) continue;
      cplx<T> *row = xbuf + p * (NX + 2);
      merge_pair<T, NX>(row, row + P, 1, row, lg, mask);
      fft_row<T, NX, true>(row, 1, twx, lg, mask);
      T *d0 = dst + (size_t)(2 * p) * NX;
      const T *a0 = addend ? addend + ((size_t)j * NZ + (size_t)r * R + 2 * p) * NX : nullptr;
      for (int n = lg; n < NX; n += G) {
        const cplx<T> z = row[n];
        T v0 = z.x * scale, v1 = z.y * scale;
        if (a0) { v0 += a0[n]; v1 += a0[NX + n]; }
        d0[n] = v0;
        d0[NX + n] = v1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// dispatch: shapes x cluster sizes instantiated here
// ---------------------------------------------------------------------------
#define IBM_CPLANE_CASES(X)                                                                     \
  X(64, 64, 2) X(96, 96, 2) X(128, 128, 2) X(128, 128, 4) X(192, 192, 4) X(256, 256, 4)        \
  X(256, 256, 8) X(384, 256, 8) X(256, 128, 4) X(128, 256, 4) X(384, 384, 8) X(512, 256, 8)

template <typename T> size_t cplane_bytes(int nx, int nz, int C) {
#define X(a, b, c) if (nx == a && nz == b && C == c) return CLayout<T, a, b, c>::fwd_bytes;
  IBM_CPLANE_CASES(X)
#undef X
  return 0;
}

template <typename T> bool cplane_supported(int nx, int nz, int C) {
  const size_t b = cplane_bytes<T>(nx, nz, C);
  return b > 0 && b <= kPlaneSmemLimit;
}

template <typename T>
cudaError_t launch_cplane_forward(const TransformGeom &g, int C, Ptr3<const T *> in, Ptr3<cplx<T> *> S,
                                  const cplx<T> *twx, const cplx<T> *twz, T in_scale, cudaStream_t st) {
#define X(a, b, c)                                                                              \
  if (g.nx == a && g.nz == b && C == c) {                                                       \
    if constexpr (CLayout<T, a, b, c>::fwd_bytes <= kPlaneSmemLimit) {                          \
      cudaError_t e = ensure_max_smem<k_cplane_fwd<T, a, b, c>>();                              \
      if (e) return e;                                                                          \
      IBM_KTRY(launch_pdl(k_cplane_fwd<T, a, b, c>, dim3(g.ny * c, g.nb), kCThreads, CLayout<T, a, b, c>::fwd_bytes, st, \
          in, S, twx, twz, in_scale, g.err, g.zrhs));                                            \
      return cudaGetLastError();                                                                \
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
    if constexpr (CLayout<T, a, b, c>::fwd_bytes <= kPlaneSmemLimit) {                          \
      cudaError_t e = ensure_max_smem<k_cplane_inv<T, a, b, c>>();                              \
      if (e) return e;                                                                          \
      IBM_KTRY(launch_pdl(k_cplane_inv<T, a, b, c>, dim3(g.ny * c, g.nb), kCThreads, CLayout<T, a, b, c>::inv_bytes, st, \
          S, out, addend, twx, twz, scale, g.err, g.zsol));                                      \
      return cudaGetLastError();                                                                \
    }                                                                                           \
  }
  IBM_CPLANE_CASES(X)
#undef X
  return cudaErrorNotSupported;
}

template size_t cplane_bytes<float>(int, int, int);
template size_t cplane_bytes<double>(int, int, int);
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
