// dft_tc.cu -- x-z plane transforms of short planes (nx, nz in {8, 16, 24,
// 32, 48, 64}) as dense DFT matrix products on the tensor cores, for FP32
// plans (plane mode kPlaneDft).
//
// The transforms are the same as the FFT path's (Sec. 2.3.3, S1: real DFT
// along x, complex DFT along z, unnormalised forward, inverse scaled by the
// caller), written as products with the DFT matrices:
//   forward  Y = X Fx        (x rows, real -> P = nx/2+1 complex)
//            S = Wz Y        (z columns, complex)
//   inverse  Y = conj(Wz) S  (z columns)
//            x = Re-synthesis of Y along x (weights 1, 2, ..., 2, 1)
// Every product runs on tcgen05 (kind::tf32, FP32 accumulators in tensor
// memory).  TF32 carries 11 significant bits, so each operand is split as
// hi + lo, both TF32 values (tf32_split), and a product is hi*hi + hi*lo +
// lo*hi: three MMAs per K step (relative error about 2^-22 per product).
// The tensor core rounds each MMA's sum into its FP32 accumulator, so the
// accumulation is spread over several accumulators that the epilogue adds
// in registers (mma3, acc_ld); the unrefined error then stays within a few
// times the FFT path's.
//
// One CTA owns a group of G <= min(128/nz, 128/P) consecutive y-planes
// (dft_shape), so both MMAs of a direction fit M = 128 rows:
//   forward  stage 1: rows (g, k) of the planes' x rows (G nz <= 128),
//                     N = 2 P8 columns (c, m): Y_c[g][k][m]
//            stage 2: rows (g, m) (G P <= 128), N = 2 nz columns (c', kz),
//                     K = nz per half: the Y_re half, then the Y_im half
//   inverse  stage 1: rows (g, m), N = 2 nz columns (c, k), K = nz per half
//            stage 2: rows (g, k), N = roundup(nx, 16) columns i, K = 2 P4
// The lane of an accumulator row is the thread that reads it back
// (tcgen05.ld 32x32b), so the second stage of the forward transform stores
// spectrum rows along kx from consecutive lanes (coalesced), and the data
// operand of each second stage is written to shared memory by the thread
// holding the first stage's row.
//
// Constant matrices (hi and lo, built on the host in the exact shared-memory
// layout) reach shared memory by bulk copies; the stage-2 z matrix is stored
// once as a stack of three blocks [s; c; -s] whose row windows [nz, 3nz) and
// [0, 2nz) are the two K halves' B operands (forward: [c; -s] for Y_re,
// [s; c] for Y_im; inverse stack [-s; c; s]: [c; s] for S_re, [-s; c] for
// S_im).  Data operands use a padded K-major layout (16 bytes between core
// matrices along K) so that the threads' stores spread over the banks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace ibm {

namespace {

constexpr int kDftThreads = 256;
constexpr uint32_t kLboPad = 144;  // data operands: 128-byte core matrices + 16 bytes
constexpr uint32_t kLboTab = 128;  // constant operands: dense
constexpr uint32_t kHdr = 128;     // barriers and the tensor-memory address
constexpr int kXLoads = 8;         // float4 loads of an x-row tile per thread (<= 128 rows x 16 / 256)
constexpr int kSLoads = 17;        // float2 loads of a spectrum group per thread (<= 128 x 33 / 256)
// Main accumulators (fewer when tensor memory is short).  Measured on GB300,
// relative L2 error of an unrefined FP32 Poisson solve on 64 x 24 x 64 with
// 1 / 2 / 3 main accumulators: 3.2e-6 / 1.4e-6 / 1.1e-6 (the FFT plane
// path: 3.0e-7); with every product in one accumulator: 1.0e-5.
constexpr int kMainAcc = 3;

inline int rup(int a, int b) { return (a + b - 1) / b * b; }
inline int pow2_at_least(int a) {
  int p = 32;
  while (p < a) p *= 2;
  return p;
}

bool dft_size_ok(int n) { return n == 8 || n == 16 || n == 24 || n == 32 || n == 48 || n == 64; }

}  // namespace

struct DftShape {
  int nx, nz, P, G, ngroups;
  int P8, N1;        // forward stage 1: N = 2 P8, column c * P8 + m
  int P4, Kf, Nf;    // inverse stage 2: K = 2 P4 (c * P4 + m), N = roundup(nx, 16)
  int ns;            // main accumulators (K steps dealt round robin); one more holds the hi*lo terms
  int wf, colsf;     // forward: columns per accumulator (both stages), columns allocated
  int wi, colsi;     // inverse: same
  uint32_t r1f, r2f, r3f;  // forward shared-memory regions (bytes)
  uint32_t r1i, r2i, r3i;  // inverse
};

static int dft_grid_cap();

// Planes per CTA: one while that gives at most two CTAs per SM (the chain
// of copies, MMAs and tensor-memory reads of a group is latency-bound, so
// more CTAs beat fuller MMAs), else the fewest that keep to that bound, at
// most min(128/nz, 128/P) (both MMAs of a direction within M = 128 rows).
static DftShape dft_shape(int nx, int ny, int nz) {
  DftShape d;
  d.nx = nx; d.nz = nz; d.P = nx / 2 + 1;
  const int gmax = std::min(128 / nz, 128 / d.P);
  d.G = std::max(1, std::min(gmax, (ny + dft_grid_cap() - 1) / dft_grid_cap()));
  d.ngroups = (ny + d.G - 1) / d.G;
  d.P8 = rup(d.P, 8); d.N1 = 2 * d.P8;
  d.P4 = rup(d.P, 4); d.Kf = 2 * d.P4; d.Nf = rup(nx, 16);
  d.wf = rup(std::max(d.N1, 2 * nz), 32);
  d.wi = rup(std::max(2 * nz, d.Nf), 32);
  d.ns = std::max(1, std::min(kMainAcc, 512 / std::max(d.wf, d.wi) - 1));
  d.colsf = pow2_at_least((d.ns + 1) * d.wf);
  d.colsi = pow2_at_least((d.ns + 1) * d.wi);
  // a padded data operand of 128 rows and K columns, hi + lo: 2 * 16 * (K/4) * 144 bytes
  d.r1f = 1152u * (uint32_t)std::max(nx, nz);
  d.r2f = 8u * (uint32_t)(d.N1 * nx);
  d.r3f = 8u * (uint32_t)(3 * nz * nz);
  d.r1i = 1152u * (uint32_t)std::max(nz, d.Kf);
  d.r2i = 8u * (uint32_t)(d.Nf * d.Kf);
  d.r3i = d.r3f;
  return d;
}

bool dft_tc_supported(int nx, int nz) {
  if (!dft_size_ok(nx) || !dft_size_ok(nz)) return false;
  const DftShape d = dft_shape(nx, 1, nz);
  return kHdr + d.r1f + d.r2f + d.r3f <= kPlaneSmemLimit && kHdr + d.r1i + d.r2i + d.r3i <= kPlaneSmemLimit &&
         d.colsf <= 512 && d.colsi <= 512;
}

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------

// byte offset of element (r, q) in a K-major operand (no swizzle)
__device__ __forceinline__ uint32_t kmaj(int r, int q, uint32_t lbo, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(q >> 2) * lbo + (uint32_t)(r & 7) * 16u + (uint32_t)(q & 3) * 4u;
}

__device__ __forceinline__ void put_split(unsigned char *h, unsigned char *l, uint32_t off, float x) {
  float a, b;
  tf32_split(x, a, b);
  *reinterpret_cast<float *>(h + off) = a;
  *reinterpret_cast<float *>(l + off) = b;
}

// K steps of a 3xTF32 product (one thread).  A, B: hi and lo operands with
// their LBO/SBO.  The accumulation is spread over ns + 1 accumulators of w
// columns from d_tmem: the hi*hi products of global K step gk go to
// accumulator gk % ns, all hi*lo and lo*hi products to accumulator ns.
// Each accumulator then takes few additions (the tensor core rounds every
// addition into an FP32 accumulator), and the epilogue adds the
// accumulators in FP32 registers.  gk0: global index of the first K step
// (a second K half continues the count and accumulates).
__device__ __forceinline__ void mma3(uint32_t d_tmem, uint32_t w, int ns, uint32_t ah, uint32_t al, uint32_t alb,
                                     uint32_t asb, uint32_t bh, uint32_t bl, uint32_t blb, uint32_t bsb, int ksteps,
                                     int gk0, uint32_t idesc) {
  const uint32_t dc = d_tmem + (uint32_t)ns * w;
  for (int ks = 0; ks < ksteps; ++ks) {
    const int gk = gk0 + ks;
    const uint32_t ao = (uint32_t)ks * 2u * alb, bo = (uint32_t)ks * 2u * blb;
    const uint64_t dah = tc_sdesc(ah + ao, alb, asb), dal = tc_sdesc(al + ao, alb, asb);
    const uint64_t dbh = tc_sdesc(bh + bo, blb, bsb), dbl = tc_sdesc(bl + bo, blb, bsb);
    tc_mma_tf32(dc, dah, dbl, idesc, gk == 0 ? 0u : 1u);
    tc_mma_tf32(dc, dal, dbh, idesc, 1u);
    tc_mma_tf32(d_tmem + (uint32_t)(gk % ns) * w, dah, dbh, idesc, gk < ns ? 0u : 1u);
  }
}

// Epilogue loads: n (4 or 8) columns at column col of this thread's lane,
// summed over the na main accumulators that were written and the
// correction accumulator (stride w columns).
template <int n>
__device__ __forceinline__ void acc_ld(uint32_t taddr, uint32_t w, int ns, int na, float *v) {
  float t[4][n], c[n];
#pragma unroll
  for (int a = 0; a < 4; ++a)
    if (a < na) {
      if constexpr (n == 8) tc_ld8(taddr + (uint32_t)a * w, t[a]);
      else tc_ld4(taddr + (uint32_t)a * w, t[a]);
    }
  if constexpr (n == 8) tc_ld8(taddr + (uint32_t)ns * w, c);
  else tc_ld4(taddr + (uint32_t)ns * w, c);
  tc_wait_ld();
#pragma unroll
  for (int i = 0; i < n; ++i) {
    float s = t[0][i];
#pragma unroll
    for (int a = 1; a < 4; ++a)
      if (a < na) s += t[a][i];
    v[i] = s + c[i];
  }
}

struct DftHdr {
  uint64_t bar_c;   // constant tables landed
  uint64_t bar_m;   // MMA batches completed (one phase per commit)
  uint32_t tmem;    // tensor-memory base address
};

// Prologue shared by both directions: barriers, bulk copy of the constant
// tables into [R2, R2 + bytes), tensor-memory allocation.
__device__ __forceinline__ uint32_t dft_prologue(DftHdr *hdr, unsigned char *R2, const float *tab, uint32_t bytes,
                                                 uint32_t cols) {
  if (threadIdx.x == 0) {
    mbar_init(&hdr->bar_c, 1);
    mbar_init(&hdr->bar_m, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&hdr->bar_c, bytes);
    const unsigned char *src = reinterpret_cast<const unsigned char *>(tab);
    for (uint32_t o = 0; o < bytes; o += 32768u) bulk_g2s(R2 + o, src + o, min(32768u, bytes - o), &hdr->bar_c);
  }
  if (threadIdx.x < 32) tc_alloc(&hdr->tmem, cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return hdr->tmem;
}

// Epilogue: tensor memory released by the allocating warp.  After a wait
// gave up, first wait (bounded) once more for the copies and the MMA batch
// (phase ph) that may still be in flight.
__device__ __forceinline__ void dft_epilogue(DftHdr *hdr, uint32_t tmem, uint32_t cols, bool ok, bool consts,
                                             uint32_t ph) {
  if (!ok) {
    if (threadIdx.x == 0) {
      if (!consts) mbar_wait(&hdr->bar_c, 0, nullptr);
      mbar_wait(&hdr->bar_m, ph, nullptr);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tc_dealloc(tmem, cols);
  }
}

// Forward: in (ny planes of nz x nx reals, times in_scale) -> S [ny][nz][P].
__global__ void __launch_bounds__(kDftThreads, 1)
k_dft_fwd(DftShape d, int ny, Ptr3<const float *> in_, Ptr3<float2 *> S_, const float *__restrict__ tab,
          float in_scale, double *zrhs, int *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  DftHdr *hdr = reinterpret_cast<DftHdr *>(smem);
  unsigned char *R1 = smem + kHdr, *R2 = R1 + d.r1f, *R3 = R2 + d.r2f;
  const uint32_t tmem = dft_prologue(hdr, R2, tab, d.r2f + d.r3f, (uint32_t)d.colsf);
  pdl_wait();
  const float *in = in_[blockIdx.y];
  float2 *S = S_[blockIdx.y];
  const int nx = d.nx, nz = d.nz, P = d.P, G = d.G;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = warp & 3, half = warp >> 2;
  // operand addresses and strides
  unsigned char *Ah = R1, *Al = R1 + d.r1f / 2;  // stage-1 x tile, then the stage-2 half operand
  const uint32_t sbo_x = (uint32_t)(nx / 4) * kLboPad, sbo_y = (uint32_t)(nz / 4) * kLboPad;
  const uint32_t sbo_f = (uint32_t)(nx / 4) * kLboTab, sbo_v = (uint32_t)(nz / 4) * kLboTab;
  const uint32_t sAh = smem_u32(Ah), sAl = smem_u32(Al);
  const uint32_t sFh = smem_u32(R2), sFl = sFh + d.r2f / 2;
  const uint32_t sVh = smem_u32(R3), sVl = sVh + d.r3f / 2;
  const uint32_t id1 = tc_idesc_tf32(128, d.N1), id2 = tc_idesc_tf32(128, 2 * nz);
  const uint32_t t_lane = (uint32_t)(quad * 32) << 16;
  bool ok = true, consts = false;
  uint32_t ph = 0;
  for (int grp = blockIdx.x; grp < d.ngroups && ok; grp += gridDim.x) {
    const int j0 = grp * G, gn = min(G, ny - j0);
    // x rows of the group's planes (contiguous), split into hi / lo
    {
      const int q4n = nx >> 2, tot = gn * nz * q4n;
      const float4 *src = reinterpret_cast<const float4 *>(in + (size_t)j0 * nz * nx);
      float4 xv[kXLoads];
#pragma unroll
      for (int it = 0; it < kXLoads; ++it) {
        const int e = tid + it * kDftThreads;
        if (e < tot) xv[it] = src[e];
      }
#pragma unroll
      for (int it = 0; it < kXLoads; ++it) {
        const int e = tid + it * kDftThreads;
        if (e < tot) {
          const int r = e / q4n, q4 = e - r * q4n;
          const uint32_t o = (uint32_t)(r >> 3) * sbo_x + (uint32_t)q4 * kLboPad + (uint32_t)(r & 7) * 16u;
          float4 h, l;
          tf32_split(xv[it].x * in_scale, h.x, l.x);
          tf32_split(xv[it].y * in_scale, h.y, l.y);
          tf32_split(xv[it].z * in_scale, h.z, l.z);
          tf32_split(xv[it].w * in_scale, h.w, l.w);
          *reinterpret_cast<float4 *>(Ah + o) = h;
          *reinterpret_cast<float4 *>(Al + o) = l;
        }
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (!consts) {
      ok = __syncthreads_and(mbar_wait(&hdr->bar_c, 0, err));
      consts = ok;  // a copy that did not land is waited for again in the epilogue
      if (!ok) break;
    }
    // stage 1: D1[(g,k)][(c,m)] = sum_i X[(g,k)][i] Fx[(c,m)][i]
    if (tid == 0) {
      tc_fence_after();
      mma3(tmem, (uint32_t)d.wf, d.ns, sAh, sAl, kLboPad, sbo_x, sFh, sFl, kLboTab, sbo_f, nx / 8, 0, id1);
      tc_commit(&hdr->bar_m);
    }
    ok = __syncthreads_and(mbar_wait(&hdr->bar_m, ph, err));
    if (!ok) break;
    ph ^= 1u;
    tc_fence_after();
    // this thread's stage-1 row (g, k), half c = half of its columns
    const int r1 = quad * 32 + lane, g1 = r1 / nz, k1 = r1 - g1 * nz;
    const bool v1 = r1 < gn * nz;
    float y[40];
    const int na1 = min(d.ns, nx / 8);
#pragma unroll
    for (int ch = 0; ch < 5; ++ch)
      if (ch * 8 < d.P8) acc_ld<8>(tmem + t_lane + (uint32_t)(half * d.P8 + ch * 8), (uint32_t)d.wf, d.ns, na1, y + ch * 8);
    // stage 2 in two K halves through one operand buffer: Y_re (c = 0) with
    // the V rows [nz, 3nz), then Y_im (c = 1) with the V rows [0, 2nz)
    for (int c = 0; c < 2 && ok; ++c) {
      if (half == c && v1) {
#pragma unroll
        for (int m = 0; m < 40; ++m)
          if (m < P) put_split(Ah, Al, kmaj(g1 * P + m, k1, kLboPad, sbo_y), y[m]);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t vrow = c == 0 ? (uint32_t)(nz / 8) * sbo_v : 0u;
        mma3(tmem, (uint32_t)d.wf, d.ns, sAh, sAl, kLboPad, sbo_y, sVh + vrow, sVl + vrow, kLboTab, sbo_v, nz / 8,
             c * (nz / 8), id2);
        tc_commit(&hdr->bar_m);
      }
      ok = __syncthreads_and(mbar_wait(&hdr->bar_m, ph, err));
      if (ok) ph ^= 1u;
    }
    if (!ok) break;
    tc_fence_after();
    // stage-2 rows (g, m): S[j0+g][kz][m] = (D2[.][kz], D2[.][nz + kz]); this
    // thread's half of kz
    {
      const int r2 = quad * 32 + lane, g2 = r2 / P, m2 = r2 - g2 * P;
      const bool v2 = r2 < gn * P;
      const int nh = nz / 2, kz0 = half * nh;
      float re[32], im[32];
      const int na2 = min(d.ns, nz / 4);
#pragma unroll
      for (int ch = 0; ch < 8; ++ch)
        if (ch * 4 < nh) {
          acc_ld<4>(tmem + t_lane + (uint32_t)(kz0 + ch * 4), (uint32_t)d.wf, d.ns, na2, re + ch * 4);
          acc_ld<4>(tmem + t_lane + (uint32_t)(nz + kz0 + ch * 4), (uint32_t)d.wf, d.ns, na2, im + ch * 4);
        }
      if (v2) {
        float2 *dst = S + ((size_t)(j0 + g2) * nz + kz0) * P + m2;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q < nh) dst[(size_t)q * P] = make_float2(re[q], im[q]);
        if (zrhs && m2 == 0 && half == 0) zrhs[j0 + g2] = (double)re[0];
      }
    }
    tc_fence_before();
  }
  dft_epilogue(hdr, tmem, (uint32_t)d.colsf, ok, consts, ph);
}

// Inverse: S [ny][nz][P] -> out = addend + scale * field (addend may be NULL
// or equal to out); zsol replaces S[j][0][0] by (zsol[j], 0).
__global__ void __launch_bounds__(kDftThreads, 1)
k_dft_inv(DftShape d, int ny, Ptr3<float2 *> S_, Ptr3<float *> out_, Ptr3<const float *> add_,
          const float *__restrict__ tab, float scale, const double *zsol, int *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  DftHdr *hdr = reinterpret_cast<DftHdr *>(smem);
  unsigned char *R1 = smem + kHdr, *R2 = R1 + d.r1i, *R3 = R2 + d.r2i;
  const uint32_t tmem = dft_prologue(hdr, R2, tab, d.r2i + d.r3i, (uint32_t)d.colsi);
  pdl_wait();
  const float2 *S = S_[blockIdx.y];
  float *out = out_[blockIdx.y];
  const float *add = add_[blockIdx.y];
  const int nx = d.nx, nz = d.nz, P = d.P, G = d.G, P4 = d.P4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = warp & 3, half = warp >> 2;
  unsigned char *Ah = R1, *Al = R1 + d.r1i / 2;  // stage-1 half operand, then the stage-2 operand
  const uint32_t sbo_s = (uint32_t)(nz / 4) * kLboPad, sbo_y = (uint32_t)(d.Kf / 4) * kLboPad;
  const uint32_t sbo_f = (uint32_t)(d.Kf / 4) * kLboTab, sbo_v = (uint32_t)(nz / 4) * kLboTab;
  const uint32_t sAh = smem_u32(Ah), sAl = smem_u32(Al);
  const uint32_t sFh = smem_u32(R2), sFl = sFh + d.r2i / 2;
  const uint32_t sVh = smem_u32(R3), sVl = sVh + d.r3i / 2;
  const uint32_t id1 = tc_idesc_tf32(128, 2 * nz), id2 = tc_idesc_tf32(128, d.Nf);
  const uint32_t t_lane = (uint32_t)(quad * 32) << 16;
  bool ok = true, consts = false;
  uint32_t ph = 0;
  for (int grp = blockIdx.x; grp < d.ngroups && ok; grp += gridDim.x) {
    const int j0 = grp * G, gn = min(G, ny - j0);
    // the group's spectrum (contiguous [gn][nz][P])
    const int plane = nz * P, tot = gn * plane;
    const float2 *src = S + (size_t)j0 * plane;
    float2 sv[kSLoads];
#pragma unroll
    for (int it = 0; it < kSLoads; ++it) {
      const int e = tid + it * kDftThreads;
      if (e < tot) {
        sv[it] = src[e];
        if (zsol) {
          const int g = e / plane;
          if (e == g * plane) sv[it] = make_float2((float)zsol[j0 + g], 0.f);
        }
      }
    }
    // stage 1 in two K halves: S_re with the V rows [nz, 3nz), then S_im
    // with the V rows [0, 2nz); rows (g, m), K = kz
    for (int c = 0; c < 2 && ok; ++c) {
#pragma unroll
      for (int it = 0; it < kSLoads; ++it) {
        const int e = tid + it * kDftThreads;
        if (e < tot) {
          const int g = e / plane, rem = e - g * plane, kz = rem / P, m = rem - kz * P;
          put_split(Ah, Al, kmaj(g * P + m, kz, kLboPad, sbo_s), c == 0 ? sv[it].x : sv[it].y);
        }
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (!consts) {
        ok = __syncthreads_and(mbar_wait(&hdr->bar_c, 0, err));
        consts = ok;
        if (!ok) break;
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t vrow = c == 0 ? (uint32_t)(nz / 8) * sbo_v : 0u;
        mma3(tmem, (uint32_t)d.wi, d.ns, sAh, sAl, kLboPad, sbo_s, sVh + vrow, sVl + vrow, kLboTab, sbo_v, nz / 8,
             c * (nz / 8), id1);
        tc_commit(&hdr->bar_m);
      }
      ok = __syncthreads_and(mbar_wait(&hdr->bar_m, ph, err));
      if (ok) ph ^= 1u;
    }
    if (!ok) break;
    tc_fence_after();
    // stage-1 rows (g, m) -> stage-2 operand rows (g, k), column c * P4 + m
    {
      const int r = quad * 32 + lane, g = r / P, m = r - g * P;
      const bool v = r < gn * P;
      float yv[64];
      const int na1 = min(d.ns, nz / 4);
#pragma unroll
      for (int ch = 0; ch < 8; ++ch)
        if (ch * 8 < nz) acc_ld<8>(tmem + t_lane + (uint32_t)(half * nz + ch * 8), (uint32_t)d.wi, d.ns, na1, yv + ch * 8);
      if (v) {
#pragma unroll
        for (int k = 0; k < 64; ++k)
          if (k < nz) put_split(Ah, Al, kmaj(g * nz + k, half * P4 + m, kLboPad, sbo_y), yv[k]);
      }
      // zero K padding m in [P, P4) of both halves, rows of this group
      const int npad = P4 - P, zt = gn * nz * 2 * npad;
      for (int e = tid; e < zt; e += kDftThreads) {
        const int rr = e / (2 * npad), rem = e - rr * 2 * npad, cc = rem / npad, mm = P + rem - cc * npad;
        const uint32_t o = kmaj(rr, cc * P4 + mm, kLboPad, sbo_y);
        *reinterpret_cast<float *>(Ah + o) = 0.f;
        *reinterpret_cast<float *>(Al + o) = 0.f;
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // stage 2: D[(g,k)][i] = sum_(c,m) Y_c[g][k][m] F[i][(c,m)]
    if (tid == 0) {
      tc_fence_after();
      mma3(tmem, (uint32_t)d.wi, d.ns, sAh, sAl, kLboPad, sbo_y, sFh, sFl, kLboTab, sbo_f, d.Kf / 8, 0, id2);
      tc_commit(&hdr->bar_m);
    }
    ok = __syncthreads_and(mbar_wait(&hdr->bar_m, ph, err));
    if (!ok) break;
    ph ^= 1u;
    tc_fence_after();
    {
      const int r = quad * 32 + lane;
      const bool v = r < gn * nz;
      const int nh = nx / 2, i0 = half * nh;
      float xv[32];
      const int na2 = min(d.ns, d.Kf / 8);
#pragma unroll
      for (int ch = 0; ch < 8; ++ch)
        if (ch * 4 < nh) acc_ld<4>(tmem + t_lane + (uint32_t)(i0 + ch * 4), (uint32_t)d.wi, d.ns, na2, xv + ch * 4);
      if (v) {
        const size_t row = ((size_t)j0 * nz + r) * nx + i0;
        float4 *dst = reinterpret_cast<float4 *>(out + row);
        const float4 *ad = add ? reinterpret_cast<const float4 *>(add + row) : nullptr;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q * 4 < nh) {
            float4 o = make_float4(scale * xv[4 * q], scale * xv[4 * q + 1], scale * xv[4 * q + 2],
                                   scale * xv[4 * q + 3]);
            if (ad) {
              const float4 a = ad[q];
              o.x += a.x; o.y += a.y; o.z += a.z; o.w += a.w;
            }
            dst[q] = o;
          }
      }
    }
    tc_fence_before();
  }
  dft_epilogue(hdr, tmem, (uint32_t)d.colsi, ok, consts, ph);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

// nearest TF32 value (ties to even) of a float
float tf32_round_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// A dense K-major operand of R rows and K columns, hi then lo, at tab[base].
struct TabWriter {
  std::vector<float> &tab;
  size_t base;
  int R, K;
  void put(int r, int q, double v) {
    const size_t o = (size_t)(r / 8) * (K / 4) * 32 + (size_t)(q / 4) * 32 + (r % 8) * 4 + (q % 4);
    const float h = tf32_round_host((float)v);
    tab[base + o] = h;
    tab[base + (size_t)R * K + o] = tf32_round_host((float)(v - (double)h));
  }
};

}  // namespace

// Host tables: forward [Fx hi, lo | V hi, lo], inverse [Fi hi, lo | V' hi, lo].
static void dft_tables(int nx, int nz, std::vector<float> &fwd, std::vector<float> &inv) {
  const DftShape d = dft_shape(nx, 1, nz);
  const int P = d.P;
  fwd.assign((d.r2f + d.r3f) / 4, 0.f);
  inv.assign((d.r2i + d.r3i) / 4, 0.f);
  const double tp = 2.0 * M_PI;
  // forward x: row c * P8 + m, column i: cos(2 pi i m / nx), -sin(...)
  TabWriter fx{fwd, 0, d.N1, nx};
  for (int m = 0; m < P; ++m)
    for (int i = 0; i < nx; ++i) {
      const double a = tp * (double)((long)i * m % nx) / nx;
      fx.put(m, i, std::cos(a));
      fx.put(d.P8 + m, i, -std::sin(a));
    }
  // z stacks: forward [s; c; -s], inverse [-s; c; s], s[r][k] = sin(2 pi r k / nz)
  TabWriter vf{fwd, (size_t)d.r2f / 4, 3 * nz, nz};
  TabWriter vi{inv, (size_t)d.r2i / 4, 3 * nz, nz};
  for (int r = 0; r < nz; ++r)
    for (int k = 0; k < nz; ++k) {
      const double a = tp * (double)((long)r * k % nz) / nz;
      const double s = std::sin(a), c = std::cos(a);
      vf.put(r, k, s); vf.put(nz + r, k, c); vf.put(2 * nz + r, k, -s);
      vi.put(r, k, -s); vi.put(nz + r, k, c); vi.put(2 * nz + r, k, s);
    }
  // inverse x: row i, column c * P4 + m: w_m cos(2 pi i m / nx), -w_m sin(...)
  TabWriter fi{inv, 0, d.Nf, d.Kf};
  for (int i = 0; i < nx; ++i)
    for (int m = 0; m < P; ++m) {
      const double w = (m == 0 || 2 * m == nx) ? 1.0 : 2.0;
      const double a = tp * (double)((long)i * m % nx) / nx;
      fi.put(i, m, w * std::cos(a));
      fi.put(i, d.P4 + m, -w * std::sin(a));
    }
}

cudaError_t dft_tc_upload(int nx, int nz, void **fwd, void **inv, size_t *bytes) {
  std::vector<float> f, i;
  dft_tables(nx, nz, f, i);
  *fwd = *inv = nullptr;
  cudaError_t e = cudaMalloc(fwd, f.size() * 4);
  if (e != cudaSuccess) { *fwd = nullptr; return e; }
  e = cudaMalloc(inv, i.size() * 4);
  if (e != cudaSuccess) { cudaFree(*fwd); *fwd = *inv = nullptr; return e; }
  e = cudaMemcpy(*fwd, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(*inv, i.data(), i.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(*fwd); cudaFree(*inv); *fwd = *inv = nullptr; return e; }
  *bytes = (f.size() + i.size()) * 4;
  return cudaSuccess;
}

static int dft_grid_cap() {
  static int cap = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? 2 * sms : 304;
  }();
  return cap;
}

cudaError_t launch_dft_forward(const TransformGeom &g, Ptr3<const float *> in, Ptr3<float2 *> S, float in_scale,
                               cudaStream_t st) {
  if (!g.dft_fwd || !dft_tc_supported(g.nx, g.nz)) return cudaErrorNotSupported;
  const DftShape d = dft_shape(g.nx, g.ny, g.nz);
  IBM_KTRY(ensure_max_smem<k_dft_fwd>());
  const dim3 grid((unsigned)std::min(d.ngroups, dft_grid_cap()), (unsigned)g.nb);
  return launch_pdl(k_dft_fwd, grid, dim3(kDftThreads), kHdr + d.r1f + d.r2f + d.r3f, st, d, g.ny, in, S,
                    (const float *)g.dft_fwd, in_scale, g.zrhs, g.err);
}

cudaError_t launch_dft_inverse(const TransformGeom &g, Ptr3<float2 *> S, Ptr3<float *> out,
                               Ptr3<const float *> addend, float scale, cudaStream_t st) {
  if (!g.dft_inv || !dft_tc_supported(g.nx, g.nz)) return cudaErrorNotSupported;
  const DftShape d = dft_shape(g.nx, g.ny, g.nz);
  IBM_KTRY(ensure_max_smem<k_dft_inv>());
  const dim3 grid((unsigned)std::min(d.ngroups, dft_grid_cap()), (unsigned)g.nb);
  return launch_pdl(k_dft_inv, grid, dim3(kDftThreads), kHdr + d.r1i + d.r2i + d.r3i, st, d, g.ny, S, out, addend,
                    (const float *)g.dft_inv, scale, g.zsol, g.err);
}

}  // namespace ibm
