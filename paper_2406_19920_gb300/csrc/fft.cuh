// fft.cuh -- shared-memory mixed-radix FFT run by a group of lanes of one warp.
//
// A length-N complex transform is done in Stockham autosort passes of radix
// 2, 3, 4 or 8 (N = 2^a 3^b, b <= 1).  Pass p with radix R and stride Ns
// (the product of the earlier radices) takes butterfly b in [0, N/R): it
// reads x[b + r N/R], r < R, multiplies input r by W_N^{(b mod Ns) r N/(Ns R)},
// applies the radix-R DFT in registers and writes output r to
// ((b / Ns) Ns R + b mod Ns) + r Ns.  After the last pass the data are in
// natural order.  The group of G lanes owns one row; every lane holds
// E = N/G values in registers, so a pass reads all, syncs the warp, writes
// all and syncs again -- in place, with no second buffer.
//
// Twiddles W_N^m = exp(-2 pi i m / N) come from a table built on the host in
// FP64 and rounded once to the working precision.
#pragma once

#include "common.cuh"

namespace ibm {

// Lanes per row (G) and radix of each pass for every supported length.
// G * E = N; each radix divides E so that every lane runs E/R butterflies.
template <int N> struct FftPlan;
#define IBM_FFT_PLAN(N_, G_, R0, R1, R2, R3)                                   \
  template <> struct FftPlan<N_> {                                            \
    static constexpr int G = G_;                                              \
    static constexpr int E = N_ / G_;                                         \
    __host__ __device__ static constexpr int radix(int p) {                   \
      return p == 0 ? R0 : p == 1 ? R1 : p == 2 ? R2 : p == 3 ? R3 : 0;        \
    }                                                                          \
  };
IBM_FFT_PLAN(8, 1, 8, 0, 0, 0)
IBM_FFT_PLAN(12, 1, 3, 4, 0, 0)
IBM_FFT_PLAN(16, 2, 4, 4, 0, 0)
IBM_FFT_PLAN(24, 2, 3, 4, 2, 0)
IBM_FFT_PLAN(32, 4, 8, 4, 0, 0)
IBM_FFT_PLAN(48, 4, 3, 4, 4, 0)
IBM_FFT_PLAN(64, 8, 8, 8, 0, 0)
IBM_FFT_PLAN(96, 4, 3, 8, 4, 0)
IBM_FFT_PLAN(128, 16, 8, 4, 4, 0)
IBM_FFT_PLAN(192, 16, 3, 4, 4, 4)
IBM_FFT_PLAN(256, 32, 8, 8, 4, 0)
IBM_FFT_PLAN(384, 16, 3, 8, 8, 2)
IBM_FFT_PLAN(512, 32, 8, 8, 8, 0)
#undef IBM_FFT_PLAN

// ---------------------------------------------------------------------------
// radix-R DFTs in registers; INV selects the +i sign (unnormalised inverse)
// ---------------------------------------------------------------------------
template <bool INV, typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
  C t = a; a = cadd(t, b); b = csub(t, b);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C &a0, C &a1, C &a2) {
  using T = decltype(a0.x);
  const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
  C s = cadd(a1, a2), d = csub(a1, a2);
  C m; m.x = a0.x - (T)0.5 * s.x; m.y = a0.y - (T)0.5 * s.y;
  a0 = cadd(a0, s);
  // forward: X1 = m - i h d, X2 = m + i h d
  C ihd; ihd.x = -h * d.y; ihd.y = h * d.x;  // +i h d
  if (INV) { a1 = cadd(m, ihd); a2 = csub(m, ihd); }
  else     { a1 = csub(m, ihd); a2 = cadd(m, ihd); }
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  C t3 = cmul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2); a2 = csub(t0, t2);
  a1 = cadd(t1, t3); a3 = csub(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C *v) {
  using T = decltype(v[0].x);
  const T s = (T)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= W8^k (fwd: exp(-i pi k / 4))
  C w1, w3;
  if (INV) {
    w1.x = s * (o1.x - o1.y); w1.y = s * (o1.x + o1.y);      // (1+i)/sqrt2
    w3.x = -s * (o3.x + o3.y); w3.y = s * (o3.x - o3.y);     // (-1+i)/sqrt2
  } else {
    w1.x = s * (o1.x + o1.y); w1.y = s * (o1.y - o1.x);      // (1-i)/sqrt2
    w3.x = s * (o3.y - o3.x); w3.y = -s * (o3.x + o3.y);     // (-1-i)/sqrt2
  }
  C w2 = cmul_mi<INV>(o2);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1); v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2); v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3); v[7] = csub(e3, w3);
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C *v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
}

// ---------------------------------------------------------------------------
// One row transform by the G lanes of a group.
//   row:    first element in shared memory; element n at row[n * stride]
//   tw:     W_N^m, m in [0, N), in shared memory
//   lg:     lane index inside the group, in [0, G)
//   mask:   lanes of the warp taking part (all of them run the same passes)
// ---------------------------------------------------------------------------
template <typename T, int N, bool INV, int P, int NS>
__device__ __forceinline__ void fft_pass(cplx<T> *row, int stride, const cplx<T> *tw, int lg,
                                         unsigned mask) {
  constexpr int R = FftPlan<N>::radix(P);
  if constexpr (R != 0) {
    constexpr int G = FftPlan<N>::G;
    constexpr int E = FftPlan<N>::E;
    constexpr int NB = E / R;
    static_assert(E % R == 0, "radix must divide the per-lane element count");
    cplx<T> v[E];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = lg + G * q;
      const int k = b % NS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cplx<T> x = row[(b + r * (N / R)) * stride];
        if (NS > 1 && r > 0) {
          const cplx<T> w = tw[k * r * (N / (NS * R))];
          x = INV ? cmulc(x, w) : cmul(x, w);
        }
        v[q * R + r] = x;
      }
      dft<R, INV>(&v[q * R]);
    }
    __syncwarp(mask);
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = lg + G * q;
      const int k = b % NS;
      const int d = (b / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) row[(d + r * NS) * stride] = v[q * R + r];
    }
    __syncwarp(mask);
    fft_pass<T, N, INV, P + 1, NS * R>(row, stride, tw, lg, mask);
  }
}

template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_row(cplx<T> *row, int stride, const cplx<T> *tw, int lg,
                                        unsigned mask) {
  fft_pass<T, N, INV, 0, 1>(row, stride, tw, lg, mask);
}

// Copy a twiddle table (N entries) from global to shared memory.
template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T> *dst, const cplx<T> *src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// real row pairs: rows a, b are transformed together as z = a + i b
// ---------------------------------------------------------------------------

// After fft_row on z = a + i b (row[0..N)), write the half spectra:
// A to dstA[k*ds], B to dstB[k*ds], k = 0..N/2.  Reads everything first.
template <typename T, int N>
__device__ __forceinline__ void split_pair(cplx<T> *row, cplx<T> *dstA, cplx<T> *dstB, int ds, int lg,
                                           unsigned mask) {
  constexpr int G = FftPlan<N>::G;
  constexpr int H = N / 2 + 1;
  constexpr int KT = (H + G - 1) / G;
  cplx<T> A[KT], B[KT];
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int k = lg + G * t;
    if (k < H) {
      const cplx<T> zk = row[k];
      const cplx<T> zn = row[(N - k) % N];
      A[t] = mk<T>((T)0.5 * (zk.x + zn.x), (T)0.5 * (zk.y - zn.y));
      // D = zk - conj(zn); B = -i D / 2
      B[t] = mk<T>((T)0.5 * (zk.y + zn.y), (T)-0.5 * (zk.x - zn.x));
    }
  }
  __syncwarp(mask);
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int k = lg + G * t;
    if (k < H) {
      dstA[k * ds] = A[t];
      dstB[k * ds] = B[t];
    }
  }
  __syncwarp(mask);
}

// Build Z_k = A_k + i B_k (k = 0..N-1, Hermitian extension) into row[0..N).
// A at srcA[k*ss], B at srcB[k*ss]; the imaginary parts of the k = 0 and
// k = N/2 bins are dropped as a real inverse transform does.
template <typename T, int N>
__device__ __forceinline__ void merge_pair(const cplx<T> *srcA, const cplx<T> *srcB, int ss, cplx<T> *row,
                                           int lg, unsigned mask) {
  constexpr int G = FftPlan<N>::G;
  constexpr int H = N / 2 + 1;
  constexpr int KT = (H + G - 1) / G;
  cplx<T> A[KT], B[KT];
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int k = lg + G * t;
    if (k < H) {
      A[t] = srcA[k * ss];
      B[t] = srcB[k * ss];
      if (k == 0 || k == N / 2) { A[t].y = 0; B[t].y = 0; }
    }
  }
  __syncwarp(mask);
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int k = lg + G * t;
    if (k < H) {
      row[k] = mk<T>(A[t].x - B[t].y, A[t].y + B[t].x);
      if (k > 0 && k < N / 2) row[N - k] = mk<T>(A[t].x + B[t].y, B[t].x - A[t].y);
    }
  }
  __syncwarp(mask);
}

}  // namespace ibm
