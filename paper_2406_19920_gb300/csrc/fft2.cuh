// fft2.cuh -- register-resident DFTs and the two-step row transform.
//
// A length-N transform is split as N = N1 * N2 (both even).  With
// n = n1 + N1 n2 and k = k2 + N2 k1,
//   X[k2 + N2 k1] = sum_n1 W_N1^{n1 k1} W_N^{n1 k2} sum_n2 W_N2^{n2 k2} x[n1 + N1 n2],
// so step 1 is a length-N2 DFT held in the registers of one thread (one per
// n1), step 2 multiplies by W_N^{n1 k2}, and step 3 is a length-N1 DFT per
// k2, after one exchange of the N values through shared memory.  The first
// step reads its inputs straight from global memory and the last one writes
// its outputs straight back: each element crosses shared memory once.
//
// The in-register DFTs of composite size use the same factorisation with
// compile-time twiddles W_M^m = exp(-2 pi i m / M), which come from
// compile-time cos/sin below (the fraction m / M is reduced to the first
// octant with the exact symmetries of the circle, then the Taylor series
// are summed in double precision and rounded once to the working type).
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace ibm {

namespace ctrig {
struct CS {
  double c, s;
};
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
__host__ __device__ constexpr double sin_series(double x) {
  double term = x, sum = x;
  for (int k = 1; k <= 12; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cos_series(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k <= 12; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// (cos, sin) of 2 pi p / q turns, 0 <= p < q
__host__ __device__ constexpr CS cs_frac(long p, long q) {
  if (2 * p >= q) {  // t = pi + u
    const CS r = cs_frac(2 * p - q, 2 * q);
    return {-r.c, -r.s};
  }
  if (4 * p >= q) {  // t = pi/2 + u
    const CS r = cs_frac(4 * p - q, 4 * q);
    return {-r.s, r.c};
  }
  if (8 * p > q) {  // t = pi/2 - u, u < pi/4
    const CS r = cs_frac(q - 4 * p, 4 * q);
    return {r.s, r.c};
  }
  const double x = kTwoPi * (double)p / (double)q;
  return {cos_series(x), sin_series(x)};
}
__host__ __device__ constexpr CS cs_turn(long m, long n) {
  long p = m % n;
  if (p < 0) p += n;
  return cs_frac(p, n);
}
}  // namespace ctrig

template <int I, int E, typename F> __device__ __forceinline__ void static_for(F &&f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, E>(f);
  }
}

// x * W_N^M (forward, W = exp(-2 pi i / N)) or x * conj(W_N^M) (inverse)
template <bool INV, int M, int N, typename C> __device__ __forceinline__ C twiddle_const(C x) {
  using T = decltype(x.x);
  constexpr int m = ((M % N) + N) % N;
  if constexpr (m == 0) {
    return x;
  } else if constexpr (2 * m == N) {
    return mk<T>(-x.x, -x.y);
  } else if constexpr (4 * m == N) {
    return cmul_mi<INV>(x);
  } else if constexpr (4 * m == 3 * N) {
    return cmul_mi<!INV>(x);
  } else {
    constexpr ctrig::CS w = ctrig::cs_turn(m, N);
    const T c = (T)w.c, s = (T)w.s;
    if (INV) return mk<T>(x.x * c - x.y * s, x.y * c + x.x * s);
    return mk<T>(x.x * c + x.y * s, x.y * c - x.x * s);
  }
}

template <bool INV, int N, typename C> __device__ __forceinline__ void reg_dft(C *v);

// v[0..R*M) in natural order -> DFT in natural order (R M = N)
template <bool INV, int R, int M, typename C> __device__ __forceinline__ void reg_dft_ct(C *v) {
  constexpr int N = R * M;
  C y[N];
  static_for<0, R>([&](auto i1) {
    constexpr int n1 = decltype(i1)::value;
    C t[M];
#pragma unroll
    for (int n2 = 0; n2 < M; ++n2) t[n2] = v[n1 + R * n2];
    reg_dft<INV, M>(t);
    static_for<0, M>([&](auto i2) {
      constexpr int k2 = decltype(i2)::value;
      y[n1 * M + k2] = twiddle_const<INV, n1 * k2, N>(t[k2]);
    });
  });
#pragma unroll
  for (int k2 = 0; k2 < M; ++k2) {
    C u[R];
#pragma unroll
    for (int n1 = 0; n1 < R; ++n1) u[n1] = y[n1 * M + k2];
    reg_dft<INV, R>(u);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) v[k2 + M * k1] = u[k1];
  }
}

template <bool INV, int N, typename C> __device__ __forceinline__ void reg_dft(C *v) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (N == 3) {
    dft3<INV>(v[0], v[1], v[2]);
  } else if constexpr (N == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 8) {
    dft8<INV>(v);
  } else if constexpr (N == 6) {
    reg_dft_ct<INV, 2, 3>(v);
  } else if constexpr (N == 12) {
    reg_dft_ct<INV, 4, 3>(v);
  } else if constexpr (N == 16) {
    reg_dft_ct<INV, 4, 4>(v);
  } else if constexpr (N == 24) {
    reg_dft_ct<INV, 8, 3>(v);
  } else if constexpr (N == 32) {
    reg_dft_ct<INV, 4, 8>(v);
  } else {
    static_assert(N == 0, "no register DFT of this size");
  }
}

// Factorisation of each supported length: N1 lanes of step 1 per row (each a
// length-N2 register DFT), N2 length-N1 DFTs in step 3.
template <int N> struct TwoStep;
#define IBM_TWO_STEP(N_, N1_)                     \
  template <> struct TwoStep<N_> {                \
    static constexpr int N1 = N1_;                \
    static constexpr int N2 = N_ / N1_;           \
    static_assert(N1 % 2 == 0 && N2 % 2 == 0, ""); \
  };
IBM_TWO_STEP(8, 2)
IBM_TWO_STEP(12, 2)
IBM_TWO_STEP(16, 4)
IBM_TWO_STEP(24, 4)
IBM_TWO_STEP(32, 4)
IBM_TWO_STEP(48, 4)
IBM_TWO_STEP(64, 8)
IBM_TWO_STEP(96, 8)
IBM_TWO_STEP(128, 8)
IBM_TWO_STEP(192, 8)
IBM_TWO_STEP(256, 16)
IBM_TWO_STEP(384, 16)
IBM_TWO_STEP(512, 16)
#undef IBM_TWO_STEP

// Step-2 twiddles in shared memory, laid out [k2][n1] so that the N1 lanes of
// step 1 read consecutive entries: tw2[k2 * N1 + n1] = W_N^{n1 k2}, gathered
// from the plan's table tw[m] = W_N^m (n1 k2 < N).
template <typename T, int N>
__device__ __forceinline__ void load_step_twiddles(cplx<T> *tw2, const cplx<T> *__restrict__ tw) {
  constexpr int N1 = TwoStep<N>::N1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int k2 = i / N1, n1 = i - k2 * N1;
    tw2[i] = tw[n1 * k2];
  }
}


// ---------------------------------------------------------------------------
// Steps of the two-step transform for the three access patterns.  X is the
// exchange buffer in shared memory; sources and destinations may be global
// or shared memory.
// ---------------------------------------------------------------------------

// Rows forward, step 1, lane n1 of one real row pair (a = rows[0, N),
// b = rows[N, 2N)): z = s (a + i b); x = the lane's exchange row (N2 entries).
template <typename T, int N>
__device__ __forceinline__ void rfwd_step1(const T *rows, T s, int n1, const cplx<T> *tw2, cplx<T> *x) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  cplx<T> v[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) v[n2] = mk<T>(rows[n1 + N1 * n2] * s, rows[N + n1 + N1 * n2] * s);
  reg_dft<false, N2>(v);
  x[0] = v[0];
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) x[k2] = cmul(v[k2], tw2[k2 * N1 + n1]);
}

// Rows forward, step 3, job q in [0, N2/2] of one pair (xp: the pair's
// exchange rows, pitch PITCH): the columns q and N2 - q give Z_k and Z_{N-k}
// together; writes A_k to dA[k] and B_k to dB[k] for its k <= N/2.
template <typename T, int N, int PITCH>
__device__ __forceinline__ void rfwd_step3(const cplx<T> *xp, int q, cplx<T> *dA, cplx<T> *dB) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  const T h = (T)0.5;
  auto put = [&](int k, cplx<T> zk, cplx<T> zn) {
    dA[k] = mk<T>(h * (zk.x + zn.x), h * (zk.y - zn.y));
    dB[k] = mk<T>(h * (zk.y + zn.y), -h * (zk.x - zn.x));
  };
  cplx<T> u[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) u[n1] = xp[n1 * PITCH + q];
  reg_dft<false, N1>(u);
  if (q == 0) {  // k = N2 k1, partner N2 (N1 - k1)
#pragma unroll
    for (int k1 = 0; k1 <= N1 / 2; ++k1) put(N2 * k1, u[k1], u[(N1 - k1) % N1]);
  } else if (q == N2 / 2) {  // k = N2/2 + N2 k1, partner N2/2 + N2 (N1 - 1 - k1)
#pragma unroll
    for (int k1 = 0; k1 < N1 / 2; ++k1) put(q + N2 * k1, u[k1], u[N1 - 1 - k1]);
  } else {
    cplx<T> w[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) w[n1] = xp[n1 * PITCH + (N2 - q)];
    reg_dft<false, N1>(w);
#pragma unroll
    for (int k1 = 0; k1 < N1 / 2; ++k1) {
      put(q + N2 * k1, u[k1], w[N1 - 1 - k1]);
      put(N2 - q + N2 * k1, w[k1], u[N1 - 1 - k1]);
    }
  }
}

// Rows inverse, step 1, lane n1: Z_n = A_n + i B_n from the half spectra
// sA, sB (n <= N/2; imaginary parts of bins 0 and N/2 dropped) and their
// Hermitian extension for n > N/2.
template <typename T, int N>
__device__ __forceinline__ void rinv_step1(const cplx<T> *sA, const cplx<T> *sB, int n1, const cplx<T> *tw2,
                                           cplx<T> *x) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  cplx<T> v[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    const int n = n1 + N1 * n2;
    if (n <= N / 2) {
      cplx<T> a = sA[n], b = sB[n];
      if (n == 0 || n == N / 2) { a.y = (T)0; b.y = (T)0; }
      v[n2] = mk<T>(a.x - b.y, a.y + b.x);
    } else {
      const cplx<T> a = sA[N - n], b = sB[N - n];
      v[n2] = mk<T>(a.x + b.y, b.x - a.y);
    }
  }
  reg_dft<true, N2>(v);
  x[0] = v[0];
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) x[k2] = cmulc(v[k2], tw2[k2 * N1 + n1]);
}

// Rows inverse, step 3, job k2 of one pair: row a gets scale Re z (+ aa),
// row b scale Im z (+ ab), at k2 + N2 k1.  Addends may alias the outputs.
template <typename T, int N, int PITCH>
__device__ __forceinline__ void rinv_step3(const cplx<T> *xp, int k2, T *da, T *db, const T *aa, const T *ab,
                                           T scale) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  // the addend's loads go out first and land while the DFT runs
  T a0[N1], a1[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    a0[k1] = aa ? aa[k2 + N2 * k1] : (T)0;
    a1[k1] = aa ? ab[k2 + N2 * k1] : (T)0;
  }
  cplx<T> u[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) u[n1] = xp[n1 * PITCH + k2];
  reg_dft<true, N1>(u);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    const int k = k2 + N2 * k1;
    da[k] = fma(u[k1].x, scale, a0[k1]);
    db[k] = fma(u[k1].y, scale, a1[k1]);
  }
}

// Columns, step 1, lane n1 of one column; at(n1, n2) points at element
// n1 + N1 n2 of the column (so a column may be spread over several CTAs'
// shared memory); x = X + n1 N2 W + c (the column's entries W apart).  With
// sub0, element 0 is replaced by v0 before transforming.
template <typename T, int N, bool INV, int W, typename At>
__device__ __forceinline__ void col_step1_at(At at, int n1, const cplx<T> *tw2, cplx<T> *x, bool sub0, cplx<T> v0) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  cplx<T> v[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) v[n2] = *at(n1, n2);
  if (sub0 && n1 == 0) v[0] = v0;
  reg_dft<INV, N2>(v);
  x[0] = v[0];
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) {
    const cplx<T> w = tw2[k2 * N1 + n1];
    x[k2 * W] = INV ? cmulc(v[k2], w) : cmul(v[k2], w);
  }
}

// Columns, step 3, job (c, k2): writes element k2 + N2 k1 to *at(k2, k1);
// returns the k1 = 0 output (bin k2).
template <typename T, int N, bool INV, int W, typename At>
__device__ __forceinline__ cplx<T> col_step3_at(const cplx<T> *X, int c, int k2, At at) {
  constexpr int N1 = TwoStep<N>::N1, N2 = TwoStep<N>::N2;
  cplx<T> u[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) u[n1] = X[(n1 * N2 + k2) * W + c];
  reg_dft<INV, N1>(u);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) *at(k2, k1) = u[k1];
  return u[0];
}

// The same for a column of stride `stride` from `col`.
template <typename T, int N, bool INV, int W>
__device__ __forceinline__ void col_step1(const cplx<T> *col, size_t stride, int n1, const cplx<T> *tw2, cplx<T> *x,
                                          bool sub0, cplx<T> v0) {
  constexpr int N1 = TwoStep<N>::N1;
  col_step1_at<T, N, INV, W>([&](int a, int b) { return col + (size_t)(a + N1 * b) * stride; }, n1, tw2, x, sub0,
                             v0);
}
template <typename T, int N, bool INV, int W>
__device__ __forceinline__ cplx<T> col_step3(const cplx<T> *X, int c, int k2, cplx<T> *col, size_t stride) {
  constexpr int N2 = TwoStep<N>::N2;
  return col_step3_at<T, N, INV, W>(X, c, k2, [&](int a, int b) { return col + (size_t)(a + N2 * b) * stride; });
}

}  // namespace ibm
