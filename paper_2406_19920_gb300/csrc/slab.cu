// slab.cu -- the fused direct solve for FP32 wall-bounded grids whose
// (y, z) slabs fit a thread-block cluster (Sec. 2.3.3, S1.1 + S1.2 / S2.1 +
// S2.2, the same method as the split passes in three global passes):
//
//   1. x rows forward (k_rows_fwd_t): every real row pair -> half spectra,
//      written kx-major, S[kx][y][z], so that one kx slab [y][z] is
//      contiguous;
//   2. slab (k_slab): a cluster of C CTAs per kx, CTA r holding the 32 rows
//      y in [32 r, 32 r + 32) of the slab in shared memory (one bulk copy
//      each half): the forward z transform of every row, the tridiagonal
//      solve along y of every kz pencil as the segmented two-ended sweep of
//      k_pencil_seg with one 32-row segment per CTA (the per-segment
//      carries cross the cluster through distributed shared memory), the
//      FP64 zero mode in the kx = 0 cluster, the inverse z transform, and
//      one bulk copy back per half;
//   3. x rows inverse (k_rows_inv_t): half spectra -> real rows, scaled by
//      1 / (nx nz), plus the optional addend.
// A refinement step adds the residual r = b - A x computed inside the
// correction's forward x rows (k_rows_fwd_res_s for 256-point rows,
// k_rows_fwd_res_t otherwise), then passes 2 and 3 again.
//
// Each pass reads and writes the field once: 24 B per point in FP32, the
// method's compulsory traffic, against 40 B for the split passes (whose z
// passes read and write the spectrum twice more).  The z transforms and the
// sweep run on data already in shared memory.
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fft2.cuh"
#include "internal.h"
#include "seg.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace ibm {

// ---------------------------------------------------------------------------
// x rows with the kx-major spectrum.  Element (kx, row) of the spectrum is at
// S[kx * rows + row] with row = y nz + z (rows = ny nz).  A CTA takes RP
// consecutive row pairs (2p, 2p + 1: the same y, consecutive z), i.e. one
// contiguous block of real rows and, for every kx, one contiguous run of
// 2 RP spectrum values.
//   forward: step 1 with lanes along n1 (the row's consecutive x, read
//            straight from global memory), the exchange [n1][k2][p] (pitch
//            QF, odd), step 3 with lanes along p so that each kx is written
//            as 2 RP consecutive values (A_k, B_k of the pair);
//   inverse: one bulk load per kx into a staging area [kx][2 RP] in shared
//            memory, step 1 with lanes along p, the exchange [p][n1][k2]
//            (pitch QI, odd), step 3 with lanes along k2 writing the rows
//            (pitch N + 16 floats: no bank conflicts) to the staging, one bulk
//            store per row, or a bulk add (FP32 reduction at the destination)
//            when the result is added to the output in place.  Read straight
//            from global memory, the 2 RP-value runs of all kx of a CTA came
//            in 20 % slower.
// ---------------------------------------------------------------------------
constexpr int kRowT = 256;

template <int N> struct RowT {
  static constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2, P = N / 2 + 1;
  static constexpr int RP = kRowT / N1 > 1 ? kRowT / N1 : 1;  // row pairs per CTA
  static constexpr int QF = N2 * RP + 1;
  static constexpr int QI = N1 * N2 + 1;
  static constexpr int POUT = N + 16;     // floats per staged row (inverse output)
  static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t stage_i = mx((size_t)P * 2 * RP * 8, (size_t)2 * RP * POUT * 4);
  static constexpr size_t smem_f = (size_t)N * 8 + (size_t)N1 * QF * 8;
  static constexpr size_t smem_r = smem_f + (size_t)2 * RP * (N + 8) * 4;  // + the residual tile
  static constexpr size_t a128(size_t b) { return (b + 127) & ~(size_t)127; }
  // inverse: where each thread has one job in both steps (N1 = N2), the
  // exchange area lies in the block's own stage (the spectrum is read into
  // registers before it is written, and it is read before the output rows
  // are), which lets three CTAs share an SM instead of two
  static constexpr bool XSTAGE = N1 == N2;
  static constexpr size_t o_stage = a128((size_t)N * 8 + (XSTAGE ? 0 : (size_t)RP * QI * 8));  // 128-byte aligned tensor-load targets
  static constexpr size_t stage_a = a128(stage_i);
  static constexpr size_t smem_i = o_stage + 2 * stage_a + 16;  // two stages
  static_assert(!XSTAGE || (size_t)RP * QI * 8 <= stage_a, "the exchange area fits a stage");
  static_assert(!XSTAGE || RP * N1 == kRowT, "one job per thread in both steps");
};

// Steps of the forward x rows of np row pairs: real rows 2 p and 2 p + 1 at
// src + 2 p pitch and src + (2 p + 1) pitch (global memory or a shared
// tile), spectra to S from pair pair0 on.
//   step 1, job (p, n1): the length-N2 DFT of the pair's entries n1 + N1 n2
//           (loaded and transformed in registers, then stored into the
//           exchange X [n1][k2][p] with the step-2 twiddles);
//   step 3, job (q, p): the columns q and N2 - q give Z_k and Z_{N-k}
//           together; the half spectra of the pair's rows are
//           A_k = (Z_k + conj Z_{N-k}) / 2 and B_k = -i (Z_k - conj Z_{N-k}) / 2
//           for k <= N/2, written as the 2 np consecutive values of each kx.
template <int N>
__device__ __forceinline__ void rows_fwd_load1(const float *src, int pitch, float in_scale, int p, int n1,
                                               float2 (&v)[TwoStep<N>::N2]) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  const float *a = src + (size_t)(2 * p) * pitch;
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) v[n2] = make_float2(a[n1 + N1 * n2] * in_scale, a[pitch + n1 + N1 * n2] * in_scale);
  reg_dft<false, N2>(v);
}
template <int N>
__device__ __forceinline__ void rows_fwd_store1(float2 *X, int p, int n1, const float2 (&v)[TwoStep<N>::N2],
                                                const float2 *tw2) {
  using Cfg = RowT<N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, RP = Cfg::RP, QF = Cfg::QF;
  float2 *x = X + n1 * QF + p;
  x[0] = v[0];
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) x[k2 * RP] = cmul(v[k2], tw2[k2 * N1 + n1]);
}
template <int N>
__device__ __forceinline__ void rows_fwd_step3(const float2 *X, float2 *__restrict__ S, int pair0, int np, int rows,
                                               int tid, int nthr) {
  using Cfg = RowT<N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, RP = Cfg::RP, QF = Cfg::QF, J3 = N2 / 2 + 1;
  for (int job = tid; job < np * J3; job += nthr) {
    const int q = job / np, p = job - q * np;
    float2 *dA = S + 2 * (size_t)(pair0 + p);
    auto put = [&](int k, float2 zk, float2 zn) {
      float2 *d = dA + (size_t)k * rows;
      d[0] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
      d[1] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    };
    float2 u[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = X[n1 * QF + q * RP + p];
    reg_dft<false, N1>(u);
    if (q == 0) {
#pragma unroll
      for (int k1 = 0; k1 <= N1 / 2; ++k1) put(N2 * k1, u[k1], u[(N1 - k1) % N1]);
    } else if (q == N2 / 2) {
#pragma unroll
      for (int k1 = 0; k1 < N1 / 2; ++k1) put(q + N2 * k1, u[k1], u[N1 - 1 - k1]);
    } else {
      float2 w[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) w[n1] = X[n1 * QF + (N2 - q) * RP + p];
      reg_dft<false, N1>(w);
#pragma unroll
      for (int k1 = 0; k1 < N1 / 2; ++k1) {
        put(q + N2 * k1, u[k1], w[N1 - 1 - k1]);
        put(N2 - q + N2 * k1, w[k1], u[N1 - 1 - k1]);
      }
    }
  }
}

// Steps 1 - 3 by the whole CTA (kRowT threads).
template <int N>
__device__ __forceinline__ void rows_fwd_steps(const float *src, int pitch, float in_scale, float2 *__restrict__ S,
                                               int pair0, int np, int rows, const float2 *tw2, float2 *X) {
  constexpr int N1 = RowT<N>::N1, N2 = RowT<N>::N2;
  for (int job = threadIdx.x; job < np * N1; job += kRowT) {
    const int p = job / N1, n1 = job - p * N1;
    float2 v[N2];
    rows_fwd_load1<N>(src, pitch, in_scale, p, n1, v);
    rows_fwd_store1<N>(X, p, n1, v, tw2);
  }
  __syncthreads();
  rows_fwd_step3<N>(X, S, pair0, np, rows, threadIdx.x, kRowT);
}

template <int N>
__global__ void __launch_bounds__(kRowT)
k_rows_fwd_t(const float *__restrict__ in, float2 *__restrict__ S, const float2 *__restrict__ tw, int npairs,
             int rows, float in_scale, int *err) {
  using Cfg = RowT<N>;
  (void)err;  // no waits: every access is a plain coalesced load or store
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);
  float2 *X = tw2 + N;  // [N1][k2][p]
  load_step_twiddles<float, N>(tw2, tw);
  pdl_wait();  // the input field is the predecessor's output
  const int pair0 = blockIdx.x * Cfg::RP;
  const int np = min(Cfg::RP, npairs - pair0);
  __syncthreads();
  rows_fwd_steps<N>(in + (size_t)pair0 * 2 * N, N, in_scale, S, pair0, np, rows, tw2, X);
}

// The refinement's correction right-hand side and its forward x rows in one
// pass: the residual r = b - A x (residual4, the slab path's wall kinds) of
// the CTA's 2 RP rows into a shared tile (pitch N + 8 floats: the two rows a
// warp reads in step 1 fall on different banks), then the forward x rows of
// the tile.  r itself never reaches global memory.  norms: the FP64 sums of
// the residual pass, when wanted.
template <int N, int BC, bool SIGMA>
__global__ void __launch_bounds__(kRowT)
k_rows_fwd_res_t(ResidualArgs A, const float *__restrict__ b, const float *__restrict__ x, float2 *__restrict__ S,
                 const float2 *__restrict__ tw, int npairs, int rows, double *norms) {
  using Cfg = RowT<N>;
  constexpr int TP = N + 8, Q4 = N / 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);
  float2 *X = tw2 + N;                                            // [N1][k2][p]
  float *tile = reinterpret_cast<float *>(X + Cfg::N1 * Cfg::QF);  // [2 RP][TP]
  load_step_twiddles<float, N>(tw2, tw);
  pdl_wait();  // x is the predecessor's output
  const int pair0 = blockIdx.x * Cfg::RP;
  const int np = min(Cfg::RP, npairs - pair0);
  // the CTA's rows lie in one y plane (2 RP divides nz on the slab path)
  const int row0 = 2 * pair0, j = row0 / A.nz, k0 = row0 - j * A.nz;
  const size_t pl = (size_t)A.nx * A.nz;
  const float *xc = x + (size_t)row0 * N, *bc = b + (size_t)row0 * N;
  const float *xlo = j > 0 ? xc - pl : nullptr, *xhi = j + 1 < A.ny ? xc + pl : nullptr;
  {  // the block's rows of b and x and x's neighbouring planes, into L2 while the first loads go out
    const uint32_t nb = (uint32_t)(2 * np) * N * 4;
    const float *pf = threadIdx.x == 0 ? bc : threadIdx.x == 1 ? xc : threadIdx.x == 2 ? xlo : xhi;
    if (threadIdx.x < 4 && pf) bulk_prefetch_l2(pf, nb);
  }
  float2 m = make_float2(0.f, 0.f);
  if (A.boff) m = *reinterpret_cast<const float2 *>(A.boff + 1);
  double r2 = 0.0, b2 = 0.0, r1 = 0.0, b1 = 0.0;
  for (int job = threadIdx.x; job < 2 * np * Q4; job += kRowT) {
    const int rr = job / Q4, i0 = 4 * (job - rr * Q4);
    float4 bt;
    const float4 res = residual4_rows<BC, SIGMA>(A, bc, xc, xlo, xhi, rr * N + i0, i0, k0 + rr, m, bt);
    if (norms) residual4_norms(res, bt, r2, b2, r1, b1);
    *reinterpret_cast<float4 *>(tile + rr * TP + i0) = res;
  }
  if (norms) block_accumulate(r2, b2, r1, b1, norms);
  __syncthreads();
  rows_fwd_steps<N>(tile, TP, 1.0f, S, pair0, np, rows, tw2, X);
}

// ---------------------------------------------------------------------------
// Streaming form of the refinement's first pass for 256-point x rows (the
// same r = b - A x and forward x rows as k_rows_fwd_res_t).
//
// A CTA takes one block of ZB = 32 consecutive z rows (z0 .. z0 + 31) and
// walks up a range of y planes ya .. yb - 1.  The x rows it needs (planes
// y - 1, y, y + 1, each with the two z neighbours z0 - 1 and z0 + 32,
// periodic in z) arrive by bulk copies in a ring of four plane slots, two
// planes ahead of their first use: every x value is read from memory once
// per CTA (plus one plane at each end of its range) instead of three times
// (once per plane that uses it), and no thread waits on a global load of x.
// Two warp groups work on consecutive planes:
//   residual group (threads 256 .. 511): r of plane y into tile buffer
//     y & 1, x from the ring, b from global memory (each quadruple of the
//     next plane into its register once the row before has used it, the
//     block into L2 two planes ahead); its first thread issues the ring's
//     copies, each as soon as the group is done with the plane the slot
//     held (x stays in L2 at evict-last priority: the correction is added
//     to it after the next pass);
//   transform group (threads 0 .. 255): the forward x rows of the buffer of
//     the plane before (step 1 reads the tile into registers, after which
//     the buffer serves as the exchange area of steps 2 and 3).
// A buffer is handed over through mbarriers (full: 256 residual arrivals,
// free: 256 transform arrivals), and so is a ring slot (sfree: 256 residual
// arrivals once the plane is read for the last time; the first residual
// thread waits for them before it reuses the slot), so that no residual warp
// waits for the others at a barrier.  Every wait is bounded; a residual warp
// that gives up leaves its loop as a whole, the transform group as a whole
// (the AND of its threads' results), the other waits then give up too, and
// the copies in flight are waited for before the CTA exits.
// ---------------------------------------------------------------------------
struct StreamCfg {
  static constexpr int N = 256, ZB = 32, SR = ZB + 2;  // x rows, rows per block, rows per ring slot
  static constexpr int TP = N + 8;                     // tile pitch (floats)
  static constexpr int GT = 256;                       // threads per warp group
  static constexpr size_t slot_bytes = (size_t)SR * N * 4;
  static constexpr size_t buf_bytes = (size_t)ZB * TP * 4;
  static constexpr size_t o_ring = 0;
  static constexpr size_t o_buf = o_ring + 4 * slot_bytes;
  static constexpr size_t o_tw = o_buf + 2 * buf_bytes;
  static constexpr size_t o_bar = o_tw + (size_t)N * 8;
  static constexpr size_t bytes = o_bar + 128;
  static_assert(buf_bytes >= (size_t)RowT<N>::N1 * RowT<N>::QF * 8, "the exchange area fits a tile buffer");
  static_assert(2 * RowT<N>::RP == ZB && RowT<N>::RP * RowT<N>::N1 == GT, "one step-1 job per transform thread");
};

template <int BC, bool SIGMA>
__global__ void __launch_bounds__(2 * StreamCfg::GT, 1)
k_rows_fwd_res_s(ResidualArgs A, const float *__restrict__ b, const float *__restrict__ x, float2 *__restrict__ S,
                 const float2 *__restrict__ tw, int rows, int kper, int *err) {
  using Cfg = StreamCfg;
  constexpr int N = Cfg::N, ZB = Cfg::ZB, SR = Cfg::SR, TP = Cfg::TP, GT = Cfg::GT;
  constexpr int N1 = RowT<N>::N1, N2 = RowT<N>::N2, RP = RowT<N>::RP;
  extern __shared__ __align__(128) unsigned char smem[];
  float *ring = reinterpret_cast<float *>(smem + Cfg::o_ring);
  unsigned char *bufs = smem + Cfg::o_buf;
  float2 *tw2 = reinterpret_cast<float2 *>(smem + Cfg::o_tw);
  uint64_t *xbar = reinterpret_cast<uint64_t *>(smem + Cfg::o_bar);  // [4] ring slots
  uint64_t *full = xbar + 4, *freeb = xbar + 6;                       // [2] each, per tile buffer
  uint64_t *sfree = xbar + 8;                                         // [4] ring slots read for the last time
  const int nz = A.nz, ny = A.ny;
  const int zb = blockIdx.x / kper, part = blockIdx.x - zb * kper;
  const int z0 = zb * ZB;
  const int ya = (int)((long)ny * part / kper), yb = (int)((long)ny * (part + 1) / kper);
  const int nsteps = yb - ya, nv = nsteps + 2;  // virtual planes v = 0 .. nv - 1 are planes ya - 1 + v
  const size_t pl = (size_t)N * nz;             // floats per y plane
  load_step_twiddles<float, N>(tw2, tw);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&xbar[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], GT);
      mbar_init(&freeb[i], GT);
    }
    for (int i = 0; i < 4; ++i) mbar_init(&sfree[i], GT);
    fence_mbar_init();
  }
  __syncthreads();
  pdl_wait();  // x is the predecessor's output
  const int t = threadIdx.x & (GT - 1);

  if (threadIdx.x >= GT) {  // ---- residual group ----
    // virtual plane v into slot v & 3, or a plain arrival where there is no
    // such plane (the wall side), so that every slot's phases stay in step
    auto issue = [&](int v) {
      const int pp = ya - 1 + v;
      uint64_t *bar = &xbar[v & 3];
      if (pp < 0 || pp >= ny) {
        mbar_arrive(bar);
        return;
      }
      float *dst = ring + (size_t)(v & 3) * SR * N;
      const float *src = x + (size_t)pp * pl;
      mbar_arrive_expect_tx(bar, (uint32_t)Cfg::slot_bytes);
      const uint64_t pol = l2_evict_last();  // (the correction is added to x after the next pass)
      bulk_g2s_hint(dst + N, src + (size_t)z0 * N, (uint32_t)ZB * N * 4, bar, pol);
      bulk_g2s_hint(dst, src + (size_t)((z0 + nz - 1) % nz) * N, N * 4, bar, pol);
      bulk_g2s_hint(dst + (size_t)(ZB + 1) * N, src + (size_t)((z0 + ZB) % nz) * N, N * 4, bar, pol);
    };
    int issued = 0;  // (thread t == 0)
    if (t == 0) {
      for (; issued < 4 && issued < nv; ++issued) issue(issued);
      for (int s = 0; s < 2 && s < nsteps; ++s)
        bulk_prefetch_l2(b + ((size_t)(ya + s) * nz + z0) * N, (uint32_t)ZB * N * 4);
    }
    float2 m = make_float2(0.f, 0.f);
    if (A.boff) m = *reinterpret_cast<const float2 *>(A.boff + 1);
    const float gs = BC == BC_NEUMANN ? 1.0f : -1.0f;
    const int lane = t & 31, c = t & 63, i0 = 4 * c, r0 = 8 * (t >> 6);  // float4 column, first of 8 rows
    // b of the thread's 8 quadruples, loaded one plane ahead: each as soon as
    // the row before has used its register, so that a load has a whole step
    // to arrive
    float4 bv[8];
    auto load_b = [&](int y) {
      const float *brow = b + ((size_t)y * nz + z0 + r0) * N + i0;
#pragma unroll
      for (int u = 0; u < 8; ++u) bv[u] = *reinterpret_cast<const float4 *>(brow + (size_t)u * N);
    };
    if (nsteps > 0) load_b(ya);
    int waited = 0;  // virtual planes seen complete
    for (int s = 0; s < nsteps; ++s) {
      const int y = ya + s, bi = s & 1;
      bool got = true;
      while (got && waited <= s + 2) {
        if (mbar_wait(&xbar[waited & 3], (uint32_t)((waited >> 2) & 1), err)) ++waited;
        else got = false;
      }
      if (got && s >= 2) got = mbar_wait(&freeb[bi], (uint32_t)(((s - 2) >> 1) & 1), err);
      if (!__all_sync(0xffffffffu, got)) break;  // warp by warp (the shuffles below want whole warps)
      if (t == 0 && s + 2 < nsteps) bulk_prefetch_l2(b + ((size_t)(y + 2) * nz + z0) * N, (uint32_t)ZB * N * 4);
      const float *sy = ring + (size_t)((s + 1) & 3) * SR * N;  // plane y
      const float *slo = ring + (size_t)(s & 3) * SR * N;       // plane y - 1
      const float *shi = ring + (size_t)((s + 2) & 3) * SR * N; // plane y + 1
      const bool lo = y > 0, hi = y + 1 < ny;
      float *tile = reinterpret_cast<float *>(bufs + bi * Cfg::buf_bytes);
      const bool bnext = s + 1 < nsteps;
      const float *bn = b + ((size_t)(y + 1) * nz + z0 + r0) * N + i0;  // b of plane y + 1
      // rows r0 - 1, r0 of the block are slot rows r0, r0 + 1
      float4 xs = *reinterpret_cast<const float4 *>(sy + r0 * N + i0);
      float4 x0 = *reinterpret_cast<const float4 *>(sy + (r0 + 1) * N + i0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = r0 + u;  // block row (z0 + r), slot row r + 1
        const float4 xn = *reinterpret_cast<const float4 *>(sy + (r + 2) * N + i0);
        const float4 g4 = make_float4(gs * x0.x, gs * x0.y, gs * x0.z, gs * x0.w);
        const float4 xd = lo ? *reinterpret_cast<const float4 *>(slo + (r + 1) * N + i0) : g4;
        const float4 xu = hi ? *reinterpret_cast<const float4 *>(shi + (r + 1) * N + i0) : g4;
        // x neighbours of the quadruple: the adjacent lanes' values, the
        // warp's end lanes from the ring (periodic x)
        float xW = __shfl_up_sync(0xffffffffu, x0.w, 1);
        float xE = __shfl_down_sync(0xffffffffu, x0.x, 1);
        if (lane == 0) xW = sy[(r + 1) * N + ((i0 + N - 1) & (N - 1))];
        if (lane == 31) xE = sy[(r + 1) * N + ((i0 + 4) & (N - 1))];
        const float2 lo2 = residual_pair<SIGMA>(
            A, make_float2(bv[u].x, bv[u].y), m, make_float2(x0.x, x0.y), make_float2(x0.y, x0.z),
            make_float2(xW, x0.x), make_float2(xn.x, xn.y), make_float2(xs.x, xs.y), make_float2(xu.x, xu.y),
            make_float2(xd.x, xd.y));
        const float2 hi2 = residual_pair<SIGMA>(
            A, make_float2(bv[u].z, bv[u].w), m, make_float2(x0.z, x0.w), make_float2(x0.w, xE),
            make_float2(x0.y, x0.z), make_float2(xn.z, xn.w), make_float2(xs.z, xs.w), make_float2(xu.z, xu.w),
            make_float2(xd.z, xd.w));
        *reinterpret_cast<float4 *>(tile + r * TP + i0) = make_float4(lo2.x, lo2.y, hi2.x, hi2.y);
        if (bnext) bv[u] = *reinterpret_cast<const float4 *>(bn + (size_t)u * N);
        xs = x0;
        x0 = xn;
      }
      mbar_arrive(&full[bi]);
      mbar_arrive(&sfree[s & 3]);  // done with plane y - 1
      bool ok = true;
      if (t == 0 && s + 4 < nv) {  // once the whole group is, its slot takes virtual plane s + 4
        ok = mbar_wait(&sfree[s & 3], (uint32_t)((s >> 2) & 1), err);
        if (ok) issue(issued++);
      }
      if (!__all_sync(0xffffffffu, ok)) break;
    }
    if (t == 0) {  // the copies still in flight (a wait gave up) land before the CTA exits
      for (int j = 0; j < 4; ++j) {
        int v = issued - 1;
        while (v >= 0 && (v & 3) != j) --v;
        if (v >= waited) mbar_wait(&xbar[j], (uint32_t)((v >> 2) & 1), nullptr);
      }
    }
  } else {  // ---- transform group ----
    const int p = t / N1, n1 = t - p * N1;  // step-1 job
    for (int s = 0; s < nsteps; ++s) {
      const int y = ya + s, bi = s & 1;
      const bool got = mbar_wait(&full[bi], (uint32_t)((s >> 1) & 1), err);
      if (!named_bar_and(2, GT, got)) break;
      float *tile = reinterpret_cast<float *>(bufs + bi * Cfg::buf_bytes);
      float2 *X = reinterpret_cast<float2 *>(tile);
      float2 v[N2];
      rows_fwd_load1<N>(tile, TP, 1.0f, p, n1, v);
      named_bar_sync(2, GT);  // every thread holds its tile values: the buffer becomes the exchange area
      rows_fwd_store1<N>(X, p, n1, v, tw2);
      named_bar_sync(2, GT);
      rows_fwd_step3<N>(X, S, (y * nz + z0) / 2, RP, rows, t, GT);
      mbar_arrive(&freeb[bi]);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kRowT)
k_rows_inv_t(const float2 *__restrict__ S, float *out, bool add, const float2 *__restrict__ tw, int npairs, int rows,
             float scale, const __grid_constant__ CUtensorMap tmap, bool use_tmap, int *err) {
  using Cfg = RowT<N>;
  constexpr int N1 = Cfg::N1, N2 = Cfg::N2, RP = Cfg::RP, QI = Cfg::QI, P = Cfg::P, POUT = Cfg::POUT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);
  float2 *Xsep = tw2 + N;                            // [p][n1][k2] (unless it lies in the stage)
  unsigned char *stage0 = smem_raw + Cfg::o_stage;  // two stages of stage_a bytes
  uint64_t *bar = reinterpret_cast<uint64_t *>(stage0 + 2 * Cfg::stage_a);
  load_step_twiddles<float, N>(tw2, tw);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  const int nblk = (npairs + RP - 1) / RP;
  __syncthreads();
  pdl_wait();  // the spectrum is the predecessor's output
  // The P runs of block blk into stage st, completion on bar[st] (thread 0
  // arms the barrier; a barrier orders that before the copies): one tensor
  // load of the [P][2 RP] box of the spectrum (whole box, the rows past a
  // partial last block read as zero), or one bulk copy per run.
  auto arm = [&](int blk, int st) {
    if (threadIdx.x == 0)
      mbar_arrive_expect_tx(&bar[st], (uint32_t)P * (use_tmap ? RP : min(RP, npairs - blk * RP)) * 16);
  };
  auto issue = [&](int blk, int st) {
    float4 *stin = reinterpret_cast<float4 *>(stage0 + st * Cfg::stage_a);
    const int pair0 = blk * RP;
    if (use_tmap) {
      if (threadIdx.x == 0) tensor_g2s_2d_hint(stin, &tmap, 4 * pair0, 0, &bar[st], l2_evict_first());
      return;
    }
    const uint32_t nb = (uint32_t)min(RP, npairs - pair0) * 16;
    const uint64_t pol = l2_evict_first();  // the spectrum is read for the last time
    for (int k = threadIdx.x; k < P; k += kRowT)
      bulk_g2s_hint(stin + k * RP, S + (size_t)k * rows + 2 * (size_t)pair0, nb, &bar[st], pol);
  };
  int blk = blockIdx.x;
  if (blk < nblk) {
    arm(blk, 0);
    __syncthreads();
    issue(blk, 0);
  }
  bool loaded_next = false;  // the other stage has copies issued (and not yet waited for)
  for (int i = 0; blk < nblk; ++i, blk += gridDim.x) {
    const int st = i & 1;
    const int nxt = blk + gridDim.x;
    // the next block's runs into the other stage, once the stores of the
    // block before this one (the other stage's output rows) have read it
    loaded_next = false;
    if (nxt < nblk) {
      if (threadIdx.x < 2 * RP) bulk_wait_read();
      arm(nxt, st ^ 1);
      __syncthreads();
      issue(nxt, st ^ 1);
      loaded_next = true;
    }
    if (!__syncthreads_and(mbar_wait(&bar[st], (uint32_t)((i >> 1) & 1), err))) {
      // copies still in flight land before the CTA's memory is reused
      mbar_wait(&bar[st], (uint32_t)((i >> 1) & 1), nullptr);
      if (loaded_next) mbar_wait(&bar[st ^ 1], (uint32_t)(((i + 1) >> 1) & 1), nullptr);
      loaded_next = false;
      break;
    }
    const float4 *stin = reinterpret_cast<const float4 *>(stage0 + st * Cfg::stage_a);  // [P][RP] (A, B) in
    float *stout = reinterpret_cast<float *>(stage0 + st * Cfg::stage_a);               // [2 RP][POUT] rows out
    float2 *X = Cfg::XSTAGE ? reinterpret_cast<float2 *>(stage0 + st * Cfg::stage_a) : Xsep;
    const int pair0 = blk * RP;
    const int np = min(RP, npairs - pair0);
    // step 1: Z_n = A_n + i B_n (imaginary parts of bins 0 and N/2 dropped)
    // and its Hermitian extension for n > N/2
    auto step1_load = [&](int n1, int p, float2 (&v)[N2]) {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int n = n1 + N1 * n2;
        if (n <= N / 2) {
          float4 ab = stin[n * RP + p];
          if (n == 0 || n == N / 2) { ab.y = 0.f; ab.w = 0.f; }
          v[n2] = make_float2(ab.x - ab.w, ab.y + ab.z);
        } else {
          const float4 ab = stin[(N - n) * RP + p];
          v[n2] = make_float2(ab.x + ab.w, ab.z - ab.y);
        }
      }
      reg_dft<true, N2>(v);
    };
    auto step1_store = [&](int n1, int p, const float2 (&v)[N2]) {
      float2 *x = X + p * QI + n1 * N2;
      x[0] = v[0];
#pragma unroll
      for (int k2 = 1; k2 < N2; ++k2) x[k2] = cmulc(v[k2], tw2[k2 * N1 + n1]);
    };
    auto step3_store = [&](int p, int k2, const float2 (&u)[N1]) {
      float *da = stout + (2 * p) * POUT, *db = da + POUT;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        da[k2 + N2 * k1] = u[k1].x * scale;
        db[k2 + N2 * k1] = u[k1].y * scale;
      }
    };
    if constexpr (Cfg::XSTAGE) {
      // one job per thread: every read of an area ends (barrier) before it
      // is overwritten: spectrum -> registers -> exchange -> registers -> rows
      const int job = threadIdx.x;
      const bool a1 = job < np * N1, a3 = job < np * N2;
      const int n1 = job / np, p1 = job - n1 * np;
      const int p3 = job / N2, k2 = job - p3 * N2;
      float2 v[N2];
      if (a1) step1_load(n1, p1, v);
      __syncthreads();
      if (a1) step1_store(n1, p1, v);
      __syncthreads();
      float2 u[N1];
      if (a3) {
#pragma unroll
        for (int q = 0; q < N1; ++q) u[q] = X[p3 * QI + q * N2 + k2];
        reg_dft<true, N1>(u);
      }
      __syncthreads();
      if (a3) step3_store(p3, k2, u);
    } else {
      for (int job = threadIdx.x; job < np * N1; job += kRowT) {
        const int n1 = job / np, p = job - n1 * np;
        float2 v[N2];
        step1_load(n1, p, v);
        step1_store(n1, p, v);
      }
      __syncthreads();
      for (int job = threadIdx.x; job < np * N2; job += kRowT) {
        const int p = job / N2, k2 = job - p * N2;
        float2 u[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) u[n1] = X[p * QI + n1 * N2 + k2];
        reg_dft<true, N1>(u);
        step3_store(p, k2, u);
      }
    }
    fence_proxy_async();
    __syncthreads();  // (also: every thread is done with X before the next block's step 1)
    if (threadIdx.x < 2 * np) {
      const int r = threadIdx.x;
      float *dst = out + (2 * (size_t)pair0 + r) * N;
      if (add) bulk_s2g_add_f32(dst, stout + r * POUT, (uint32_t)N * 4);
      else bulk_s2g_hint(dst, stout + r * POUT, (uint32_t)N * 4, l2_evict_last());  // (the residual pass reads it)
      bulk_commit();
    }
  }
  if (threadIdx.x < 2 * RP) bulk_wait_all();  // this thread's stores are complete
}

// ---------------------------------------------------------------------------
// The slab kernel.  Rows y of the slab are the unknowns of every kz pencil
// (n = ny rows, j0 = 0: Poisson and the cell-centred Helmholtz kinds).  The
// two-ended sweep splits them as k_pencil_seg does: rows 0 .. m-1 top-down,
// rows n-1 .. m+1 bottom-up, meeting at m = n/2, in 32-row segments.  CTA r
// < C/2 owns top segment r (rows 32 r ..), CTA r >= C/2 bottom segment
// C/2 + (C - 1 - r) (its rows counted from the top wall); CTA C/2 also holds
// the meeting row m as its local row 0 (its segment has 31 rows).
// ---------------------------------------------------------------------------
template <int NZ, int C> struct SlabCfg {
  static constexpr int R = 32;        // rows per CTA (one sweep segment)
  static constexpr int NY = R * C;
  static constexpr int THREADS = NZ;  // one thread per kz pencil
  static constexpr int N1 = TwoStep<NZ>::N1, N2 = TwoStep<NZ>::N2;
  static constexpr int W = THREADS / N1;  // rows per z-transform round
  static constexpr int PN = W * N2 + 1;   // exchange pitch per n1 (odd)
  static constexpr size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
  static constexpr size_t o_slab = 0;
  static constexpr size_t o_x = o_slab + al((size_t)R * NZ * 8);
  static constexpr size_t xbytes = (size_t)N1 * PN * 8 > (size_t)R * NZ * 4 ? (size_t)N1 * PN * 8 : (size_t)R * NZ * 4;
  static constexpr size_t o_tw = o_x + al(xbytes);
  static constexpr size_t o_cf = o_tw + al((size_t)NZ * 8);
  static constexpr size_t o_cb = o_cf + al((size_t)4 * NZ * 4);
  static constexpr size_t o_xm = o_cb + al((size_t)3 * NZ * 4);
  static constexpr size_t o_zm = o_xm + al((size_t)NZ * 8);
  static constexpr size_t o_bar = o_zm + al((size_t)NY * 8);
  static constexpr size_t bytes = o_bar + 128;
  static_assert(W * N1 == THREADS, "one row per N1 threads in step 1");
  static_assert((R / 2) % W == 0, "each half of the rows is whole transform rounds");
};

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync_all() {
  cluster_arrive();
  cluster_wait();
}

// W rows of `rows` (row pitch NZ) transformed along z in place: step 1 with
// thread (c, n1) (W N1 = blockDim threads), the exchange [n1][c][k2] (pitch
// PN per n1), step 3 with job (c, k2) (W N2 jobs).
template <int NZ, int W, bool INV>
__device__ __forceinline__ void zfft_rows(float2 *rows, float2 *X, const float2 *tw2) {
  constexpr int N1 = TwoStep<NZ>::N1, N2 = TwoStep<NZ>::N2, PN = W * N2 + 1;
  {
    const int c = threadIdx.x / N1, n1 = threadIdx.x - c * N1;
    const float2 *row = rows + c * NZ;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = row[n1 + N1 * n2];
    reg_dft<INV, N2>(v);
    float2 *x = X + n1 * PN + c * N2;
    x[0] = v[0];
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) {
      const float2 t = tw2[k2 * N1 + n1];
      x[k2] = INV ? cmulc(v[k2], t) : cmul(v[k2], t);
    }
  }
  __syncthreads();
  for (int job = threadIdx.x; job < W * N2; job += blockDim.x) {
    const int c = job / N2, k2 = job - c * N2;
    float2 u[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = X[n1 * PN + c * N2 + k2];
    reg_dft<INV, N1>(u);
    float2 *row = rows + c * NZ;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) row[k2 + N2 * k1] = u[k1];
  }
  __syncthreads();
}

// Persistent: cluster q of the grid's Q clusters takes the slabs kx = q,
// q + Q, ...; while it works on one slab the next one is prefetched into L2.
// Between slabs a CTA waits until the bulk store of the previous slab has
// read its shared memory, then loads the next one.  Every peer reads this
// CTA's forward carries (cf) and its zero-mode rows only between the slab's
// two cluster barriers, and its back-substitution carries (cb, with the
// segment's product of w) and the meeting row's solution (xmb, CTA C/2)
// only between the second barrier and the next slab's first, before which
// this CTA rewrites neither: one copy of each suffices.  The carries cross
// the cluster as few times as the sweep needs: each CTA reads those of the
// segments before its own in its half, and only CTA C/2 reads both halves'
// (for the meeting row).
template <int NZ, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(NZ, (NZ >= 256 ? 2 : 3))
k_slab(float2 *S, const float2 *__restrict__ twz, const float *__restrict__ lamx, const float *__restrict__ lamz,
       PencilParams pp, double *mean_out) {
  using Cfg = SlabCfg<NZ, C>;
  constexpr int R = Cfg::R, NY = Cfg::NY, W = Cfg::W, Lh = C / 2;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int q = blockIdx.x / C, Q = gridDim.x / C;
  const int tid = threadIdx.x;
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem + Cfg::o_slab);  // [R][NZ]
  float2 *X = reinterpret_cast<float2 *>(smem + Cfg::o_x);        // z-transform exchange
  float *ws = reinterpret_cast<float *>(smem + Cfg::o_x);         // [R][NZ] w of every row (after the transforms)
  float2 *tw2 = reinterpret_cast<float2 *>(smem + Cfg::o_tw);
  float *cf = reinterpret_cast<float *>(smem + Cfg::o_cf);  // [4][NZ] yhat_end.x, .y, prod w, q of the last row
  float *cb = reinterpret_cast<float *>(smem + Cfg::o_cb);  // [3][NZ] xhat at the segment's first row, prod w
  double *zr = reinterpret_cast<double *>(smem + Cfg::o_zm);  // zero mode (CTA 0 of the kx = 0 cluster): rhs,
                                                              // scratch, then solution
  float2 *xmb = reinterpret_cast<float2 *>(smem + Cfg::o_xm);  // [NZ] meeting row solution (CTA C/2)
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Cfg::o_bar);

  // plan constants before the grid-dependency wait
  load_step_twiddles<float, NZ>(tw2, twz);
  const int kz = tid;
  const float a = (float)pp.a;
  const float lz = lamz[kz];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  pdl_wait();  // the spectrum is the predecessor's output

  // segment geometry (the same for every slab)
  const bool top = rank < Lh;
  const int seg = top ? rank : Lh + (C - 1 - rank);
  const int k0 = top ? rank * R : NY - (rank + 1) * R;  // distance of my first row from its wall
  const int len = rank == Lh ? R - 1 : R;
  const int lr0 = top ? 0 : R - 1, lstep = top ? 1 : -1;  // local row of sweep row u: lr0 + lstep u
  const float sgn = pp.neg_rhs ? -1.f : 1.f;
  auto rank_of = [](int s2) { return s2 < Lh ? s2 : C - 1 - (s2 - Lh); };
  constexpr uint32_t kHalf = (uint32_t)(R / 2) * NZ * 8;

  // A wait that gives up leaves ok false: the CTA still reaches every
  // cluster barrier of every slab (its peers wait there), issues no further
  // copies and stores nothing.  fail_par remembers the phase of the slab
  // whose copies may still be in flight (fail_bar >= 0: there was one).
  bool ok = true;
  int fail_bar = -1;
  uint32_t fail_par = 0;
  for (int it = 0;; ++it) {
    const int kx = q + it * Q;
    if (kx >= pp.P) break;  // the same for the whole cluster
    const uint32_t par = (uint32_t)(it & 1);
    float2 *gslab = S + (size_t)kx * NY * NZ + (size_t)rank * R * NZ;
    // The halves of the CTA's rows are stored and reloaded one at a time:
    // the first half's copy for this slab went out during the previous
    // slab's inverse transforms (once that half's store had read it); the
    // second goes out here, once the previous slab's second half is read.
    if (tid == 0 && ok) {
      if (it == 0) {
        mbar_arrive_expect_tx(&bar[0], kHalf);
        bulk_g2s_hint(slab, gslab, kHalf, &bar[0], l2_evict_first());
      }
      bulk_wait_read();
      mbar_arrive_expect_tx(&bar[1], kHalf);
      bulk_g2s_hint(slab + (R / 2) * NZ, gslab + (R / 2) * NZ, kHalf, &bar[1], l2_evict_first());
      if (kx + Q < pp.P) bulk_prefetch_l2(gslab + (size_t)Q * NY * NZ, 2 * kHalf);  // the next slab, into L2
    }
    const float g = (float)pp.g_add + (float)pp.g_mul * (lamx[kx] + lz);
    // forward z transforms
#pragma unroll 1
    for (int r0 = 0; r0 < R; r0 += W) {
      if (r0 == 0 || r0 == R / 2) {
        const int b = r0 == 0 ? 0 : 1;
        const bool got = ok ? __syncthreads_and(mbar_wait(&bar[b], par, pp.err)) : false;
        if (ok && !got) { fail_bar = b; fail_par = par; }
        ok = ok && got;
      }
      zfft_rows<NZ, W, false>(slab + r0 * NZ, X, tw2);
    }
    const bool zm = pp.zero_mode && kx == 0;

    // forward elimination of my segment
    const bool live = !(zm && kz == 0);
    const float e0 = g + a * (float)(top ? pp.beta_s : pp.beta_e);
    float ep, D, z;
    const bool cw = __all_sync(0xffffffffu, seg_pivots<float>(a, g, e0, k0, ep, D, z)) && len == R;
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = u < len ? slab[(lr0 + lstep * u) * NZ + kz] : make_float2(0.f, 0.f);
    float *wc = ws + kz;  // w of sweep row u at wc[NZ u]
    float2 y;
    float prod, qlast;
    if (cw) seg_forward<float, R, true, true, NZ>(v, len, k0, a, g, e0, sgn, ep, D, z, wc, y, prod, qlast);
    else seg_forward_lin<R, false, NZ>(v, len, k0, a, g, e0, sgn, ep, D, z, wc, y, prod, qlast);
    cf[0 * NZ + kz] = y.x;
    cf[1 * NZ + kz] = y.y;
    cf[2 * NZ + kz] = prod;
    cf[3 * NZ + kz] = qlast;
    cluster_sync_all();  // #1: every CTA has started; every segment's carries and row m are visible

    // the carry into my segment: the segments before it in its half of the
    // sweep (at most Lh - 1 of them).  Every peer load is issued before the
    // first is used (the segments that are not needed read this CTA's own
    // copy and are left out of the fold), so the reads cost one round trip.
    float2 c = make_float2(0.f, 0.f);
    {
      constexpr int NPR = Lh > 1 ? Lh - 1 : 1;
      float pw[NPR], px[NPR], py[NPR];
#pragma unroll
      for (int j = 0; j < Lh - 1; ++j) {
        const int s2 = (top ? 0 : Lh) + j;
        const float *pcf = cluster.map_shared_rank(cf, s2 < seg ? rank_of(s2) : rank);
        pw[j] = pcf[2 * NZ + kz];
        px[j] = pcf[kz];
        py[j] = pcf[NZ + kz];
      }
#pragma unroll
      for (int j = 0; j < Lh - 1; ++j) {
        const bool in = (top ? 0 : Lh) + j < seg;
        c.x = in ? fmaf(pw[j], c.x, px[j]) : c.x;
        c.y = in ? fmaf(pw[j], c.y, py[j]) : c.y;
      }
    }
    // the meeting row, solved by CTA C/2 (its sweep ends next to it, and it
    // holds the row) and read by the others after the second barrier:
    // (g + a q^T + a q^B) x_m = sgn f_m + a (y^T_{m-1} + y^B_{m+1})
    float2 xm = make_float2(0.f, 0.f);
    if (rank == Lh) {
      float2 yT = make_float2(0.f, 0.f);
      float pw[Lh], px[Lh], py[Lh];
#pragma unroll
      for (int s2 = 0; s2 < Lh; ++s2) {
        const float *pcf = cluster.map_shared_rank(cf, rank_of(s2));
        pw[s2] = pcf[2 * NZ + kz];
        px[s2] = pcf[kz];
        py[s2] = pcf[NZ + kz];
      }
      const float qT = cluster.map_shared_rank(cf, Lh - 1)[3 * NZ + kz];
#pragma unroll
      for (int s2 = 0; s2 < Lh; ++s2) {
        yT.x = fmaf(pw[s2], yT.x, px[s2]);
        yT.y = fmaf(pw[s2], yT.y, py[s2]);
      }
      const float2 yB = make_float2(fmaf(prod, c.x, y.x), fmaf(prod, c.y, y.y));
      const float2 fm = slab[kz];
      const float rm = rcp<float>(g + a * qT + a * qlast);
      xm.x = (sgn * fm.x + a * (yT.x + yB.x)) * rm;
      xm.y = (sgn * fm.y + a * (yT.y + yB.y)) * rm;
      xmb[kz] = xm;
    }
    const float wconst = a * rcp<float>(a + ep);
    float2 x;
    if (cw) x = seg_middle<float, R, true, true, NZ>(v, len, wconst, wc, c);
    else x = seg_middle<float, R, false, false, NZ>(v, len, wconst, wc, c);
    cb[kz] = x.x;
    cb[NZ + kz] = x.y;
    cb[2 * NZ + kz] = prod;
    // the FP64 zero mode (one warp of CTA 0 of the kx = 0 cluster): its
    // right-hand side is Re of bin kz = 0 of every row (the plane sums), read
    // from the peers' slabs, which the forward sweep left untouched; then the
    // removed mean, the pin and the nullspace
    if (zm && rank == 0 && tid < 32) {
      for (int j = tid; j < NY; j += 32) zr[j] = (double)cluster.map_shared_rank(slab, j / R)[(j % R) * NZ].x;
      __syncwarp();
      zero_mode_fp64(zr, zr, zr, NY, pp.inv_ny, pp.hy2, pp.inv_nxnz, mean_out);  // solution over the rhs
    }
    cluster_sync_all();  // #2: every segment's xhat and the zero mode's solution are visible

    // x after my last row (towards the meeting row): the meeting row folded
    // back through the segments between it and mine (at most Lh - 1; every
    // peer load issued before the first is used), then my rows stored
    {
      const float2 xmr = rank == Lh ? xm : cluster.map_shared_rank(xmb, Lh)[kz];
      const int send = top ? Lh : C;  // segments seg + 1 .. send - 1 lie between
      constexpr int NPR = Lh > 1 ? Lh - 1 : 1;
      float pw[NPR], px[NPR], py[NPR];
#pragma unroll
      for (int j = 0; j < Lh - 1; ++j) {
        const int s2 = send - 1 - j;
        const float *pcb = cluster.map_shared_rank(cb, s2 > seg ? rank_of(s2) : rank);
        pw[j] = pcb[2 * NZ + kz];
        px[j] = pcb[kz];
        py[j] = pcb[NZ + kz];
      }
      c = xmr;
#pragma unroll
      for (int j = 0; j < Lh - 1; ++j) {
        const bool in = send - 1 - j > seg;
        c.x = in ? fmaf(pw[j], c.x, px[j]) : c.x;
        c.y = in ? fmaf(pw[j], c.y, py[j]) : c.y;
      }
    }
    float2 *col = slab + lr0 * NZ + kz;
    if (cw) seg_store<float, R, true, true, NZ>(v, len, wconst, wc, c, live, col, (long)lstep * NZ);
    else seg_store<float, R, false, false, NZ>(v, len, wconst, wc, c, live, col, (long)lstep * NZ);
    if (rank == Lh && live) slab[kz] = xm;
    if (zm && tid < R) slab[tid * NZ] = make_float2((float)cluster.map_shared_rank(zr, 0)[rank * R + tid], 0.f);
    __syncthreads();

    // inverse z transforms; each half stored as soon as it is done, and the
    // next slab's first half copied in once its store has read the buffer
    // (under the second half's transforms)
#pragma unroll 1
    for (int r0 = 0; r0 < R; r0 += W) {
      zfft_rows<NZ, W, true>(slab + r0 * NZ, X, tw2);
      if (r0 + W == R / 2 || r0 + W == R) {
        const int h = r0 + W == R ? 1 : 0;
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && ok) {
          bulk_s2g_hint(gslab + h * (R / 2) * NZ, slab + h * (R / 2) * NZ, kHalf, l2_evict_last());  // (the inverse x rows read it)
          bulk_commit();
          if (h == 0 && kx + Q < pp.P) {
            bulk_wait_read();
            mbar_arrive_expect_tx(&bar[0], kHalf);
            bulk_g2s_hint(slab, gslab + (size_t)Q * NY * NZ, kHalf, &bar[0], l2_evict_first());
          }
        }
      }
    }
  }
  if (tid == 0) {
    if (ok) {
      bulk_wait_all();  // the last slab's store is complete
    } else if (fail_bar >= 0) {  // both halves of the failed slab's copies may still be in flight
      mbar_wait(&bar[0], fail_par, nullptr);
      mbar_wait(&bar[1], fail_par, nullptr);
    }
  }
  __syncthreads();
  cluster_sync_all();  // the peers have finished reading this CTA's memory
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
#define IBM_SLAB_ROWS_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

bool slab_supported(int nx, int ny, int nz) {
  (void)nx;
  return (nz == 64 || nz == 128 || nz == 256) && (ny == 64 || ny == 128 || ny == 256);
}

template <int NZ, int C>
static cudaError_t launch_slab_kernel(const PencilParams &pp, float2 *S, const float2 *twz, const float *lamx,
                                      const float *lamz, double *mean_out, cudaStream_t st) {
  using Cfg = SlabCfg<NZ, C>;
  {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
      err = cudaFuncSetAttribute(k_slab<NZ, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::bytes);
    });
    if (err != cudaSuccess) return err;
  }
  // as many clusters as can be resident at once (every one loops over its
  // share of the P slabs), and never more clusters than slabs
  static std::once_flag once_q;
  static int resident = 0;
  std::call_once(once_q, [] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * 1024);
    cfg.blockDim = dim3(Cfg::THREADS);
    cfg.dynamicSmemBytes = Cfg::bytes;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_slab<NZ, C>, &cfg) == cudaSuccess) resident = n;
    cudaGetLastError();
  });
  const int Q = resident > 0 ? std::min(resident, pp.P) : pp.P;
  IBM_KTRY(launch_pdl(k_slab<NZ, C>, dim3(Q * C), dim3(Cfg::THREADS), Cfg::bytes, st, S, twz, lamx, lamz, pp,
                      mean_out));
  return cudaGetLastError();
}

// CTAs of kernel K resident at once on the device (the grid of the
// persistent x-rows kernels).  Set the kernel's shared-memory attribute
// first.
template <auto K> static int resident_ctas(size_t smem, int threads) {
  static std::once_flag once;
  static int n = 0;
  std::call_once(once, [&] {
    int per = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, threads, smem) == cudaSuccess)
      n = per * sms;
    cudaGetLastError();
  });
  return n;
}

bool slab_residual_fused(int nx, int nz) {
  int rows = 0;  // rows a CTA of the x-rows passes takes
#define X(N) \
  if (nx == N) rows = 2 * RowT<N>::RP;
  IBM_SLAB_ROWS_N(X)
#undef X
  return rows > 0 && nx % 4 == 0 && nz % rows == 0;
}

// The inverse x rows' view of the kx-major spectrum for tensor loads: S as a
// [P][rows] array of complex values (2 floats), box [P][2 RP complex].
// false where the box does not fit the tensor unit's limits (P > 256) or
// the CUDA driver has no tensor-map encoder: the kernel then issues one bulk
// copy per run.
static bool spectrum_tmap(CUtensorMap *tm, const float2 *S, int P, int rows, int rp) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cudaGetLastError();
  });
  std::memset(tm, 0, sizeof *tm);
  if (!encode || P > 256 || 4 * rp > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows * 2, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)rows * 8};  // bytes between kx rows
  const cuuint32_t box[2] = {(cuuint32_t)(4 * rp), (cuuint32_t)P};
  const cuuint32_t estr[2] = {1, 1};
  return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(S), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N, int B, bool SG>
static cudaError_t launch_rows_fwd_res(const ResidualArgs &A, const float *b, const float *x, float2 *S,
                                       const float2 *twx, int npairs, int rows, double *norms, cudaStream_t st) {
  constexpr auto kern = k_rows_fwd_res_t<N, B, SG>;
  {  // its own size: the kernel also has static shared memory (the norm sums)
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RowT<N>::smem_r);
    });
    IBM_KTRY(err);
  }
  IBM_KTRY(launch_pdl(kern, dim3(ceil_div(npairs, RowT<N>::RP)), dim3(kRowT), RowT<N>::smem_r, st, A, b, x, S, twx,
                      npairs, rows, norms));
  return cudaGetLastError();
}

template <int B, bool SG>
static cudaError_t launch_rows_fwd_res_stream(const ResidualArgs &A, const float *b, const float *x, float2 *S,
                                              const float2 *twx, int rows, int *err, cudaStream_t st) {
  constexpr auto kern = k_rows_fwd_res_s<B, SG>;
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  static int sms = 0;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StreamCfg::bytes);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  IBM_KTRY(e);
  // one CTA per SM: every block of 32 z rows gets the same number of CTAs,
  // each a contiguous range of at least 4 y planes
  const int nzb = A.nz / StreamCfg::ZB;
  const int kper = std::max(1, std::min(sms / nzb, A.ny / 4));
  IBM_KTRY(launch_pdl(kern, dim3(nzb * kper), dim3(2 * StreamCfg::GT), StreamCfg::bytes, st, A, b, x, S, twx, rows,
                      kper, err));
  return cudaGetLastError();
}

// Whether the streaming form of the refinement's first pass takes the
// shape: 256-point x rows, z in blocks of 32 (IBM_RES_STREAM=0 keeps the
// block form everywhere).
static bool stream_residual_applies(int nx, int ny, int nz) {
  const char *e = getenv("IBM_RES_STREAM");
  return !(e && atoi(e) == 0) && nx == 256 && nz % 32 == 0 && ny >= 1;
}

cudaError_t launch_slab_residual_forward(const StencilCoef &c, int nx, int ny, int nz, const float *b, const float *x,
                                         float2 *S, const float2 *twx, const double *boff, double *norms, int *err,
                                         cudaStream_t st) {
  if (nx % 4 != 0 || ((uintptr_t)b | (uintptr_t)x) & 15u) return cudaErrorInvalidValue;
  if (c.bc != BC_NEUMANN && c.bc != BC_CELL_DIRICHLET) return cudaErrorInvalidValue;  // the slab path's kinds
  if (!slab_residual_fused(nx, nz)) return cudaErrorInvalidValue;
  const ResidualArgs A = make_args(nx, ny, nz, c, boff);
  const bool sg = c.sigma != 0.0, neu = c.bc == BC_NEUMANN;
  const int npairs = ny * nz / 2, rows = ny * nz;
  if (!norms && stream_residual_applies(nx, ny, nz)) {
    if (neu) return sg ? launch_rows_fwd_res_stream<BC_NEUMANN, true>(A, b, x, S, twx, rows, err, st)
                       : launch_rows_fwd_res_stream<BC_NEUMANN, false>(A, b, x, S, twx, rows, err, st);
    return sg ? launch_rows_fwd_res_stream<BC_CELL_DIRICHLET, true>(A, b, x, S, twx, rows, err, st)
              : launch_rows_fwd_res_stream<BC_CELL_DIRICHLET, false>(A, b, x, S, twx, rows, err, st);
  }
#define X(N)                                                                                                    \
  if (nx == N) {                                                                                                \
    if (neu) return sg ? launch_rows_fwd_res<N, BC_NEUMANN, true>(A, b, x, S, twx, npairs, rows, norms, st)      \
                       : launch_rows_fwd_res<N, BC_NEUMANN, false>(A, b, x, S, twx, npairs, rows, norms, st);    \
    return sg ? launch_rows_fwd_res<N, BC_CELL_DIRICHLET, true>(A, b, x, S, twx, npairs, rows, norms, st)        \
              : launch_rows_fwd_res<N, BC_CELL_DIRICHLET, false>(A, b, x, S, twx, npairs, rows, norms, st);      \
  }
  IBM_SLAB_ROWS_N(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_slab_solve(const PencilParams &pp, int nx, const float *in, float2 *S, float *out,
                              const float *addend, const float2 *twx, const float2 *twz, const float *lamx,
                              const float *lamz, double *mean_out, float scale, cudaStream_t st, int phase) {
  const int ny = pp.ny, nz = pp.nz;
  const int npairs = ny * nz / 2, rows = ny * nz;
  if (phase == 0) {
    bool done = false;
#define X(N)                                                                                               \
  if (nx == N) {                                                                                           \
    IBM_KTRY(ensure_max_smem<k_rows_fwd_t<N>>());                                                          \
    IBM_KTRY(launch_pdl(k_rows_fwd_t<N>, dim3(ceil_div(npairs, RowT<N>::RP)), dim3(kRowT), RowT<N>::smem_f, \
                        st, in, S, twx, npairs, rows, 1.0f, pp.err));                                       \
    done = true;                                                                                           \
  }
    IBM_SLAB_ROWS_N(X)
#undef X
    return done ? cudaGetLastError() : cudaErrorInvalidValue;
  }
  if (phase == 1) {
    const int C = ny / 32;
#define S_(NZ_, C_) \
  if (nz == NZ_ && C == C_) return launch_slab_kernel<NZ_, C_>(pp, S, twz, lamx, lamz, mean_out, st);
    S_(64, 2) S_(64, 4) S_(64, 8) S_(128, 2) S_(128, 4) S_(128, 8) S_(256, 2) S_(256, 4) S_(256, 8)
#undef S_
    return cudaErrorInvalidValue;
  }
  if (addend && addend != out) return cudaErrorInvalidValue;  // the inverse adds in place only
  bool done = false;
#define X(N)                                                                                               \
  if (nx == N) {                                                                                           \
    IBM_KTRY(ensure_max_smem<k_rows_inv_t<N>>());                                                          \
    const int nblk = ceil_div(npairs, RowT<N>::RP);                                                        \
    const int res = resident_ctas<k_rows_inv_t<N>>(RowT<N>::smem_i, kRowT);                                 \
    CUtensorMap tm;                                                                                        \
    const bool use_tm = spectrum_tmap(&tm, S, RowT<N>::P, rows, RowT<N>::RP);                               \
    IBM_KTRY(launch_pdl(k_rows_inv_t<N>, dim3(res > 0 ? std::min(nblk, res) : nblk), dim3(kRowT), RowT<N>::smem_i, \
                        st, S, out, addend != nullptr, twx, npairs, rows, scale, tm, use_tm, pp.err));      \
    done = true;                                                                                           \
  }
  IBM_SLAB_ROWS_N(X)
#undef X
  return done ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace ibm
