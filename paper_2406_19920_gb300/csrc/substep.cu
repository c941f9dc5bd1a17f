// substep.cu -- one RK stage of Eq. 2a-2h (ibm_substep).
//
// Order of work (the paper's flowchart for one stage, Sec. 2.3):
//   E1  explicit terms: du = u^e - u^{n-1}
//         = dt [(a+b) nu L u - (a+b) G p - gamma N(u) - zeta N^{n-2}]   (Eq. 2a)
//       and N(u) stored for the next stage's zeta term;
//   L2  marker positions / surface velocity at the stage start time;
//   L1  U^e = interp(u^{n-1} + du) (Eq. 2b), F = (U^d - U^e)/dt (Eq. 2c),
//       du += dt spread(F) (Eq. 2d);
//   S1  three Helmholtz solves.  Eq. 2e, (I - c L) u* = u^e - c L u^{n-1} +
//       dt f with c = beta dt nu, is solved in increment form
//       (I - c L) delta = du, u* = u^{n-1} + delta (same system: subtract
//       (I - c L) u^{n-1} from both sides); u* overwrites u;
//   E2  b = D u* / ((a+b) dt)                                          (Eq. 2f)
//   S2  Poisson solve L phi = b (refined on the FP32 path)
//   E3  u^n = u* - (a+b) dt G phi, p^n = p + phi - c L phi             (Eq. 2g, 2h)
// RK coefficients: Rai & Moin's low-storage scheme, which the paper cites
// without printing.  Advection is the conservative MAC form div(u u) with
// two-point averages (the paper names second-order central differences).
#include <cmath>

#include "plan.h"

namespace ibm {

template <typename T>
cudaError_t launch_interp(const ibm_plan_s *p, int n, const T *X, const T *u, const T *v, const T *w,
                          const T *du, const T *dv, const T *dw, T *U, const T *Ud, double inv_dt, T *F,
                          const T *X0, T *Xout, T *Udout, int kind, const double *params, double t,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_spread(const ibm_plan_s *p, int n, const T *X, const T *F, const T *dV, T *fu, T *fv, T *fw,
                          double scale, cudaStream_t st);

static const double kAlpha[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
static const double kBeta[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
static const double kGamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double kZeta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

struct Geo {
  int nx, ny, nz;
  double ihx, ihy, ihz;  // 1/h
};

// field accessor with periodic x, z
template <typename T> struct F3 {
  const T *f;
  int nx, nz;
  __device__ __forceinline__ T at(int j, int k, int i) const {
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    return f[((size_t)j * nz + k) * nx + i];
  }
};

// E1, all three components.  A CTA owns a TX x TZ column tile and marches
// up JC planes of y; the planes j-1, j, j+1 of u, v, w (and j of p) sit in a
// shared-memory ring with a one-cell periodic halo in x and z, so every
// field is read from HBM about once (plus halo and the two extra planes per
// chunk) and every stencil point comes from shared memory.  Wall rules in
// y: u, w cell-centred with the no-slip ghost (-value) in the Laplacian and
// zero wall flux in the advective y-flux; v on faces, zero at the walls
// (j = 0 stored as the wall, j = ny not stored).
//
// IO: the inflow-outflow walls of Sec. 3 instead.  The y = 0 face carries
// v = v_lo with u = w = 0 there (the ghost -value and the zero y-flux of
// u, w are unchanged; v's lower neighbour at j = 1 is v_lo); the y = Ly
// wall carries the outlet planes uo, wo (u, w at the wall: ghost 2 g - u in
// the Laplacian, flux v_face * g) and vo (v on the outlet face), [nz][nx].
constexpr int kExTX = 32, kExTZ = 8, kExJC = 16;

template <typename T, bool IO>
__global__ void __launch_bounds__(kExTX * kExTZ)
k_explicit(Geo g, const T *__restrict__ u_, const T *__restrict__ v_, const T *__restrict__ w_,
           const T *__restrict__ p_, T *Nu, T *Nv, T *Nw, T *__restrict__ du, T *__restrict__ dv,
           T *__restrict__ dw, T c_visc, T c_pres, T gam, T zet, T dt, T v_lo, const T *__restrict__ uo,
           const T *__restrict__ vo, const T *__restrict__ wo) {
  pdl_wait();
  constexpr int TX = kExTX, TZ = kExTZ, HX = TX + 2, HZ = TZ + 2, PL = HX * HZ, NT = TX * TZ;
  constexpr int NL = (PL + NT - 1) / NT;  // plane elements each thread loads
  __shared__ T su[3 * PL], sv[3 * PL], sw[3 * PL], sp[2 * PL];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * TX + tx;
  const int i0 = blockIdx.x * TX, k0 = blockIdx.y * TZ;
  const int jb = blockIdx.z * kExJC, je = min(ny, jb + kExJC);
  const int plane = nz * nx;  // < 2^31 for every supported grid
  // halo-tile element -> offset inside a plane (periodic x, z), fixed for all planes
  int off[NL];
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    const int e = tid + q * NT;
    const int hz = e / HX, hx = e - hz * HX;
    const int kk = ((k0 - 1 + hz) % nz + nz) % nz, ii = ((i0 - 1 + hx) % nx + nx) % nx;
    off[q] = e < PL ? kk * nx + ii : -1;
  }
  // a plane's tile elements of this thread: fetched into registers one
  // iteration ahead, stored into the ring after the iteration's compute
  auto fetch = [&](const T *F, int jj, T (&r)[NL]) {
    const bool ok = jj >= 0 && jj < ny;
    const T *src = F + (size_t)(ok ? jj : 0) * plane;
#pragma unroll
    for (int q = 0; q < NL; ++q) r[q] = (ok && off[q] >= 0) ? src[off[q]] : (T)0;
  };
  auto put = [&](const T (&r)[NL], T *buf) {
#pragma unroll
    for (int q = 0; q < NL; ++q)
      if (off[q] >= 0) buf[tid + q * NT] = r[q];
  };
  // ring slots of the planes j-1, j, j+1 (rotated each plane, no modulo)
  int sm = 0, s0 = PL, sp1 = 2 * PL;
  {
    T r[NL];
    fetch(u_, jb - 1, r); put(r, su + sm);
    fetch(v_, jb - 1, r); put(r, sv + sm);
    fetch(w_, jb - 1, r); put(r, sw + sm);
    fetch(u_, jb, r); put(r, su + s0);
    fetch(v_, jb, r); put(r, sv + s0);
    fetch(w_, jb, r); put(r, sw + s0);
    fetch(u_, jb + 1, r); put(r, su + sp1);
    fetch(v_, jb + 1, r); put(r, sv + sp1);
    fetch(w_, jb + 1, r); put(r, sw + sp1);
    fetch(p_, jb, r); put(r, sp);
  }
  __syncthreads();
  const int i = i0 + tx, k = k0 + tz;
  const bool inside = i < nx && k < nz;
  const int c = (tz + 1) * HX + (tx + 1);  // this column in a halo tile
  const int col = k * nx + i;
  T p_prev = (inside && jb > 0) ? p_[(size_t)(jb - 1) * plane + col] : (T)0;
  const T ihx = (T)g.ihx, ihy = (T)g.ihy, ihz = (T)g.ihz;
  const T ihx2 = ihx * ihx, ihy2 = ihy * ihy, ihz2 = ihz * ihz;
  // Every advective flux is a product of two two-point averages,
  // (a + b)/2 * (c + d)/2: the exact factor 1/4 is carried by the inverse
  // spacings it is multiplied with (q* = ih* / 4), which leaves each term's
  // rounding unchanged.
  const T qx = ihx * (T)0.25, qy = ihy * (T)0.25, qz = ihz * (T)0.25;
  const bool n_prev = zet != (T)0;  // N^{n-2} unused (and maybe unset) at stage 1
  int pb = 0;                       // P ring slot of plane j (0 or PL)
  for (int j = jb; j < je; ++j) {
    T ru[NL], rv[NL], rw[NL], rp[NL];
    const bool more = j + 1 < je;
    if (more) {
      fetch(u_, j + 2, ru);
      fetch(v_, j + 2, rv);
      fetch(w_, j + 2, rw);
      fetch(p_, j + 1, rp);
    }
    if (inside) {
      const T *Um = su + sm + c, *Uc = su + s0 + c, *Up = su + sp1 + c;
      const T *Vc = sv + s0 + c, *Vm = sv + sm + c, *Vp = sv + sp1 + c;
      const T *Wm = sw + sm + c, *Wc = sw + s0 + c, *Wp = sw + sp1 + c;
      const T *Pc = sp + pb + c;
      const bool lo = j == 0, hi = j + 1 >= ny;
      const size_t idx = (size_t)j * plane + col;
      // tile neighbours: B[dk * HX + di] relative to this column
      const T p0 = Pc[0];
      const T u0 = Uc[0], v0 = Vc[0], w0 = Wc[0];
      // outlet wall values at this column (IO, top row only)
      T ug = 0, wg = 0, vgo = 0, vgw = 0, vgs = 0;
      if (IO && hi) {
        const int iw = i == 0 ? nx - 1 : i - 1, ks = k == 0 ? nz - 1 : k - 1;
        ug = uo[col]; wg = wo[col]; vgo = vo[col];
        vgw = vo[k * nx + iw]; vgs = vo[ks * nx + i];
      }
      // ---------------- u (x-faces) ----------------
      {
        const T ue = Uc[1], uw = Uc[-1], un = Uc[HX], us = Uc[-HX];
        const T uup = Up[0], udn = Um[0];
        const T uu = hi ? (IO ? 2 * ug - u0 : -u0) : uup, ud = lo ? -u0 : udn;
        const T lap = (ue - 2 * u0 + uw) * ihx2 + (un - 2 * u0 + us) * ihz2 + (uu - 2 * u0 + ud) * ihy2;
        const T uc = u0 + ue, ucm = uw + u0;  // twice the averages
        const T txx = (uc * uc - ucm * ucm) * qx;
        // y-flux at the faces j (zero at the wall j = 0) and j+1 (zero at j+1 = ny), times 4
        const T fy0 = lo ? (T)0 : (Vc[-1] + v0) * (udn + u0);
        const T fy1 = hi ? (IO ? (vgw + vgo) * (ug + ug) : (T)0) : (Vp[-1] + Vp[0]) * (u0 + uup);
        const T fz0 = (Wc[-1] + w0) * (us + u0);
        const T fz1 = (Wc[HX - 1] + Wc[HX]) * (u0 + un);
        const T N = txx + (fy1 - fy0) * qy + (fz1 - fz0) * qz;
        const T G = (p0 - Pc[-1]) * ihx;
        const T np = n_prev ? Nu[idx] : (T)0;
        du[idx] = dt * (c_visc * lap - c_pres * G - gam * N - zet * np);
        Nu[idx] = N;
      }
      // ---------------- w (z-faces) ----------------
      {
        const T we = Wc[1], ww = Wc[-1], wn = Wc[HX], ws = Wc[-HX];
        const T wup = Wp[0], wdn = Wm[0];
        const T wu = hi ? (IO ? 2 * wg - w0 : -w0) : wup, wd = lo ? -w0 : wdn;
        const T lap = (we - 2 * w0 + ww) * ihx2 + (wn - 2 * w0 + ws) * ihz2 + (wu - 2 * w0 + wd) * ihy2;
        const T wc = w0 + wn, wcm = ws + w0;
        const T tzz = (wc * wc - wcm * wcm) * qz;
        const T fx0 = (Uc[-HX] + u0) * (ww + w0);
        const T fx1 = (Uc[1 - HX] + Uc[1]) * (w0 + we);
        const T fy0 = lo ? (T)0 : (Vc[-HX] + v0) * (wdn + w0);
        const T fy1 = hi ? (IO ? (vgs + vgo) * (wg + wg) : (T)0) : (Vp[-HX] + Vp[0]) * (w0 + wup);
        const T N = tzz + (fx1 - fx0) * qx + (fy1 - fy0) * qy;
        const T G = (p0 - Pc[-HX]) * ihz;
        const T np = n_prev ? Nw[idx] : (T)0;
        dw[idx] = dt * (c_visc * lap - c_pres * G - gam * N - zet * np);
        Nw[idx] = N;
      }
      // ---------------- v (y-faces, interior j = 1..ny-1) ----------------
      if (lo) {
        dv[idx] = (T)0;
        Nv[idx] = (T)0;
      } else {
        const T ve = Vc[1], vw = Vc[-1], vn = Vc[HX], vs = Vc[-HX];
        const T vu = hi ? (IO ? vgo : (T)0) : Vp[0], vd = j - 1 <= 0 ? (IO ? v_lo : (T)0) : Vm[0];
        const T lap = (ve - 2 * v0 + vw) * ihx2 + (vn - 2 * v0 + vs) * ihz2 + (vu - 2 * v0 + vd) * ihy2;
        const T vc = v0 + vu, vcm = vd + v0;
        const T tyy = (vc * vc - vcm * vcm) * qy;
        const T fx0 = (Um[0] + u0) * (vw + v0);
        const T fx1 = (Um[1] + Uc[1]) * (v0 + ve);
        const T fz0 = (Wm[0] + w0) * (vs + v0);
        const T fz1 = (Wm[HX] + Wc[HX]) * (v0 + vn);
        const T N = tyy + (fx1 - fx0) * qx + (fz1 - fz0) * qz;
        const T G = (p0 - p_prev) * ihy;
        const T np = n_prev ? Nv[idx] : (T)0;
        dv[idx] = dt * (c_visc * lap - c_pres * G - gam * N - zet * np);
        Nv[idx] = N;
      }
      p_prev = p0;
    }
    __syncthreads();
    if (more) {
      // plane j+2 replaces plane j-1; the ring rotates
      put(ru, su + sm);
      put(rv, sv + sm);
      put(rw, sw + sm);
      put(rp, sp + (PL - pb));
      const int t = sm;
      sm = s0; s0 = sp1; sp1 = t;
      pb = PL - pb;
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// E2: b = D u * inv_scale in plain working precision (the right-hand side of
// Eq. 2f); with dmax, additionally max |D u| evaluated exactly: float-float
// differences for FP32 fields, FP64 for FP64 fields (the projection check).
// The wall faces carry v_lo (y = 0) and v_hi ([nz][nx] at y = Ly, NULL for
// 0).
template <typename T> struct DivExact;
template <> struct DivExact<float> {
  static __device__ __forceinline__ float eval(float ue, float uw, float vn, float vs, float wt, float wb,
                                               const ff &ihx, const ff &ihy, const ff &ihz) {
    ff d = ff_mul(two_sum(ue, -uw), ihx);
    d = ff_add(d, ff_mul(two_sum(vn, -vs), ihy));
    d = ff_add(d, ff_mul(two_sum(wt, -wb), ihz));
    return fabsf(__fadd_rn(d.hi, d.lo));
  }
};
template <> struct DivExact<double> {
  static __device__ __forceinline__ double eval(double ue, double uw, double vn, double vs, double wt, double wb,
                                                const ff &ihx, const ff &ihy, const ff &ihz) {
    return fabs((ue - uw) * (double)ihx.hi + (vn - vs) * (double)ihy.hi + (wt - wb) * (double)ihz.hi +
                ((ue - uw) * (double)ihx.lo + (vn - vs) * (double)ihy.lo + (wt - wb) * (double)ihz.lo));
  }
};

template <typename T>
__global__ void __launch_bounds__(128)
k_divergence(Geo g, const T *__restrict__ u_, const T *__restrict__ v_, const T *__restrict__ w_, T *b,
             T inv_scale, T ihx_t, T ihy_t, T ihz_t, ff ihx, ff ihy, ff ihz, double *dmax, T v_lo,
             const T *__restrict__ v_hi) {
  pdl_wait();
  int i, k, j;
  const bool inside = stencil_index(g.nx, g.nz, i, k, j);
  const size_t idx = ((size_t)j * g.nz + k) * g.nx + i;
  T mx = 0;
  if (inside) {
    const F3<T> U{u_, g.nx, g.nz}, V{v_, g.nx, g.nz}, W{w_, g.nx, g.nz};
    const T vs = j == 0 ? v_lo : V.at(j, k, i);
    const T vn = j + 1 >= g.ny ? (v_hi ? v_hi[k * g.nx + i] : (T)0) : V.at(j + 1, k, i);
    const T ue = U.at(j, k, i + 1), uw = U.at(j, k, i), wt = W.at(j, k + 1, i), wb = W.at(j, k, i);
    if (b) b[idx] = ((ue - uw) * ihx_t + (vn - vs) * ihy_t + (wt - wb) * ihz_t) * inv_scale;
    if (dmax) mx = DivExact<T>::eval(ue, uw, vn, vs, wt, wb, ihx, ihy, ihz);
  }
  if (dmax) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(full, mx, o));
    if (((threadIdx.y * blockDim.x + threadIdx.x) & 31) == 0) atomic_max_nonneg(dmax, (double)mx);
  }
}

// E3: u -= k G phi (in place), p += phi - c L phi (Neumann ghosts); the
// y = 0 face of v is set to v_lo.
template <typename T>
__global__ void __launch_bounds__(128)
k_project(Geo g, T *__restrict__ u, T *__restrict__ v, T *__restrict__ w, T *__restrict__ p,
          const T *__restrict__ phi_, T kproj, T cvisc, T v_lo) {
  pdl_wait();
  int i, k, j;
  if (!stencil_index(g.nx, g.nz, i, k, j)) return;
  const size_t idx = ((size_t)j * g.nz + k) * g.nx + i;
  const F3<T> Ph{phi_, g.nx, g.nz};
  const T ihx = (T)g.ihx, ihy = (T)g.ihy, ihz = (T)g.ihz;
  const T f0 = Ph.at(j, k, i);
  const T fw = Ph.at(j, k, i - 1), fe = Ph.at(j, k, i + 1);
  const T fs = Ph.at(j, k - 1, i), fn = Ph.at(j, k + 1, i);
  const T fd = j > 0 ? Ph.at(j - 1, k, i) : f0;
  const T fu = j + 1 < g.ny ? Ph.at(j + 1, k, i) : f0;
  u[idx] -= kproj * (f0 - fw) * ihx;
  w[idx] -= kproj * (f0 - fs) * ihz;
  if (j > 0) v[idx] -= kproj * (f0 - fd) * ihy;
  else v[idx] = v_lo;
  const T lap = (fe - 2 * f0 + fw) * ihx * ihx + (fn - 2 * f0 + fs) * ihz * ihz + (fu - 2 * f0 + fd) * ihy * ihy;
  p[idx] += f0 - cvisc * lap;
}

// FP32 versions of E2 and E3 with four consecutive x points per thread:
// float4 rows, the x neighbours from the same float4 plus one or two
// scalars, shared index arithmetic (the one-point kernels are load-latency
// bound).  Each point's arithmetic is the one-point kernel's, in the same
// order.  Grid (ceil(nz nx / 4 / 128), ny), 128 threads; nx % 4 == 0 and
// 16-byte aligned fields.
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float comp4(const float4 &a, int q) { return q == 0 ? a.x : q == 1 ? a.y : q == 2 ? a.z : a.w; }
__device__ __forceinline__ void set4(float4 &a, int q, float v) {
  if (q == 0) a.x = v; else if (q == 1) a.y = v; else if (q == 2) a.z = v; else a.w = v;
}

__global__ void __launch_bounds__(128)
k_divergence_f32v(Geo g, const float *__restrict__ u_, const float *__restrict__ v_, const float *__restrict__ w_,
                  float *b, float inv_scale, float ihx_t, float ihy_t, float ihz_t, ff ihx, ff ihy, ff ihz,
                  double *dmax, float v_lo, const float *__restrict__ v_hi) {
  pdl_wait();
  const int q4 = g.nx >> 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  float mx = 0.f;
  if (t < q4 * g.nz) {
    const int k = t / q4, i0 = 4 * (t - k * q4);
    const size_t pl = (size_t)g.nx * g.nz;
    const size_t at = (size_t)j * pl + (size_t)k * g.nx + i0;
    const float4 uc = ld4(u_ + at);
    const float uE = u_[at - i0 + (i0 + 4 == g.nx ? 0 : i0 + 4)];
    const float4 vs = j == 0 ? make_float4(v_lo, v_lo, v_lo, v_lo) : ld4(v_ + at);
    const float4 vn = j + 1 >= g.ny ? (v_hi ? ld4(v_hi + (size_t)k * g.nx + i0) : make_float4(0.f, 0.f, 0.f, 0.f))
                                    : ld4(v_ + at + pl);
    const float4 wb = ld4(w_ + at);
    const float4 wt = ld4(w_ + at + (k + 1 == g.nz ? -(long)(g.nz - 1) * g.nx : (long)g.nx));
    float4 out;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float ue = q < 3 ? comp4(uc, q + 1) : uE, uw = comp4(uc, q);
      const float vnq = comp4(vn, q), vsq = comp4(vs, q), wtq = comp4(wt, q), wbq = comp4(wb, q);
      set4(out, q, ((ue - uw) * ihx_t + (vnq - vsq) * ihy_t + (wtq - wbq) * ihz_t) * inv_scale);
      if (dmax) mx = fmaxf(mx, DivExact<float>::eval(ue, uw, vnq, vsq, wtq, wbq, ihx, ihy, ihz));
    }
    if (b) *reinterpret_cast<float4 *>(b + at) = out;
  }
  if (dmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(dmax, (double)mx);
  }
}

__global__ void __launch_bounds__(128)
k_project_f32v(Geo g, float *__restrict__ u, float *__restrict__ v, float *__restrict__ w, float *__restrict__ p,
               const float *__restrict__ phi, float kproj, float cvisc, float v_lo) {
  pdl_wait();
  const int q4 = g.nx >> 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (t >= q4 * g.nz) return;
  const int k = t / q4, i0 = 4 * (t - k * q4);
  const size_t pl = (size_t)g.nx * g.nz;
  const size_t at = (size_t)j * pl + (size_t)k * g.nx + i0;
  const float ihx = (float)g.ihx, ihy = (float)g.ihy, ihz = (float)g.ihz;
  const float4 f0 = ld4(phi + at);
  const float fW = phi[at - i0 + (i0 == 0 ? g.nx - 1 : i0 - 1)];
  const float fE = phi[at - i0 + (i0 + 4 == g.nx ? 0 : i0 + 4)];
  const float4 fs = ld4(phi + at + (k == 0 ? (long)(g.nz - 1) * g.nx : -(long)g.nx));
  const float4 fn = ld4(phi + at + (k + 1 == g.nz ? -(long)(g.nz - 1) * g.nx : (long)g.nx));
  const float4 fd = j > 0 ? ld4(phi + at - pl) : f0;
  const float4 fu = j + 1 < g.ny ? ld4(phi + at + pl) : f0;
  float4 uu = ld4(u + at), vv = ld4(v + at), ww = ld4(w + at), pp = ld4(p + at);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float c0 = comp4(f0, q);
    const float fw = q == 0 ? fW : comp4(f0, q - 1), fe = q < 3 ? comp4(f0, q + 1) : fE;
    const float fsq = comp4(fs, q), fnq = comp4(fn, q), fdq = comp4(fd, q), fuq = comp4(fu, q);
    set4(uu, q, comp4(uu, q) - kproj * (c0 - fw) * ihx);
    set4(ww, q, comp4(ww, q) - kproj * (c0 - fsq) * ihz);
    set4(vv, q, j > 0 ? comp4(vv, q) - kproj * (c0 - fdq) * ihy : v_lo);
    const float lap = (fe - 2 * c0 + fw) * ihx * ihx + (fnq - 2 * c0 + fsq) * ihz * ihz + (fuq - 2 * c0 + fdq) * ihy * ihy;
    set4(pp, q, comp4(pp, q) + (c0 - cvisc * lap));
  }
  *reinterpret_cast<float4 *>(u + at) = uu;
  *reinterpret_cast<float4 *>(v + at) = vv;
  *reinterpret_cast<float4 *>(w + at) = ww;
  *reinterpret_cast<float4 *>(p + at) = pp;
}

// E2 / E3 launches: the four-point FP32 kernels, the one-point kernels for FP64.
template <typename T>
static cudaError_t launch_divergence(const Geo &g, const Launch3 &L3, const T *u, const T *v, const T *w, T *b,
                                     double inv_scale, const ff &fx, const ff &fy, const ff &fz, double *dmax, T v_lo,
                                     const T *v_hi, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    const dim3 grid((unsigned)ceil_div(g.nz * (g.nx / 4), 128), (unsigned)g.ny);
    return launch_pdl(k_divergence_f32v, grid, dim3(128), 0, st, g, u, v, w, b, (float)inv_scale, (float)g.ihx,
                      (float)g.ihy, (float)g.ihz, fx, fy, fz, dmax, v_lo, v_hi);
  } else {
    return launch_pdl(k_divergence<T>, L3.grid, L3.block, 0, st, g, u, v, w, b, (T)inv_scale, (T)g.ihx, (T)g.ihy,
                      (T)g.ihz, fx, fy, fz, dmax, v_lo, v_hi);
  }
}
template <typename T>
static cudaError_t launch_project(const Geo &g, const Launch3 &L3, T *u, T *v, T *w, T *p, const T *phi, double kproj,
                                  double cvisc, T v_lo, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    const dim3 grid((unsigned)ceil_div(g.nz * (g.nx / 4), 128), (unsigned)g.ny);
    return launch_pdl(k_project_f32v, grid, dim3(128), 0, st, g, u, v, w, p, phi, (float)kproj, (float)cvisc, v_lo);
  } else {
    return launch_pdl(k_project<T>, L3.grid, L3.block, 0, st, g, u, v, w, p, phi, (T)kproj, (T)cvisc, v_lo);
  }
}

// Outlet condition of the inflow-outflow configuration (Sec. 3):
// d phi/dt + C d phi/dy = 0 at y = Ly, advanced over the stage step
// (alpha + beta) dt by first-order upwinding from the last interior value
// (cu = step C / (hy/2) for u, w at the wall, cv = step C / hy for v's outlet
// face).  Also stores v = v_in on the inflow face (plane 0 of v) and writes
// each CTA's FP64 sum of the new outlet v to part[blockIdx.x] (fixed-order
// tree, so the total is reproducible).
constexpr int kOutT = 256;
template <typename T>
__global__ void __launch_bounds__(kOutT)
k_outflow_update(int ncol, const T *__restrict__ ul, const T *__restrict__ vl, const T *__restrict__ wl, T *uo,
                 T *vo, T *wo, T *v0, T cu, T cv, T v_in, double *part) {
  pdl_wait();
  __shared__ double ws[kOutT / 32];
  const int col = blockIdx.x * kOutT + threadIdx.x;
  double s = 0.0;
  if (col < ncol) {
    uo[col] -= cu * (uo[col] - ul[col]);
    wo[col] -= cu * (wo[col] - wl[col]);
    const T vn = vo[col] - cv * (vo[col] - vl[col]);
    vo[col] = vn;
    v0[col] = v_in;
    s = (double)vn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kOutT / 32; ++q) t += ws[q];
    part[blockIdx.x] = t;
  }
}

// Global mass balance: the outlet v is shifted by a constant so that its
// mean equals v_in (outflow = inflow; the Poisson right-hand side then has
// zero mean).  Every CTA sums the nparts partial sums in the same order.
template <typename T>
__global__ void __launch_bounds__(kOutT)
k_outflow_shift(int ncol, T *vo, double v_in, const double *__restrict__ part, int nparts, double inv_ncol) {
  pdl_wait();
  __shared__ double ws[kOutT / 32];
  __shared__ double shift;
  double s = 0.0;
  for (int q = threadIdx.x; q < nparts; q += kOutT) s += part[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kOutT / 32; ++q) t += ws[q];
    shift = v_in - t * inv_ncol;
  }
  __syncthreads();
  const int col = blockIdx.x * kOutT + threadIdx.x;
  if (col < ncol) vo[col] = (T)((double)vo[col] + shift);
}

static ff ff_host(double v) {
  ff r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

static int ensure_substep_buffers(ibm_plan_s *p, int nmk) {
  for (int q = 0; q < 4; ++q) {
    if (!p->sub[q]) {
      cudaError_t e = cudaMalloc(&p->sub[q], p->npts * p->esz);
      if (e != cudaSuccess) { p->sub[q] = nullptr; return cuda_error(e, "substep workspace"); }
      p->bytes += p->npts * p->esz;
    }
  }
  const size_t need = (size_t)nmk * 3 * p->esz;
  if (need > p->mkcap) {
    if (p->mkbuf) { cudaFree(p->mkbuf); p->bytes -= p->mkcap; p->mkbuf = nullptr; p->mkcap = 0; }
    cudaError_t e = cudaMalloc(&p->mkbuf, need);
    if (e != cudaSuccess) { p->mkbuf = nullptr; return cuda_error(e, "marker workspace"); }
    p->mkcap = need;
    p->bytes += need;
  }
  return IBM_OK;
}

template <typename T>
static int substep_t(ibm_plan_s *p, ibm_state *s, const ibm_inout *io, int stage, double dt, double nu,
                     ibm_markers *mk, cudaStream_t st, ibm_info *info) {
  const int n = stage - 1;
  const double a = kAlpha[n], b = kBeta[n], gm = kGamma[n], zt = kZeta[n];
  const double ab = a + b;
  const double cH = b * dt * nu;  // Helmholtz coefficient of Eq. 2e
  const int nmk = mk ? mk->n : 0;
  int rc = ensure_substep_buffers(p, nmk);
  if (rc) return rc;
  Geo g{p->nx, p->ny, p->nz, 1.0 / p->h[0], 1.0 / p->h[1], 1.0 / p->h[2]};
  T *u = (T *)s->u, *v = (T *)s->v, *w = (T *)s->w, *pr = (T *)s->p;
  T *du = (T *)p->sub[0], *dv = (T *)p->sub[1], *dw = (T *)p->sub[2], *phi = (T *)p->sub[3];
  T *rhs = (T *)p->bsave;
  const Launch3 L3 = stencil_launch(p->nx, p->ny, p->nz);
  InfoTrace trace(p, info != nullptr);
  if (info) {
    IBM_CUDA_TRY(cudaMemsetAsync(p->dsc + 8, 0, 2 * sizeof(double), st));
    IBM_CUDA_TRY(cudaEventRecord(p->ev0, st));
  }
  // inflow-outflow walls: outlet values advanced to the end of the stage
  // and made mass-conserving; they are the wall data of the whole stage
  const T v_lo = io ? (T)io->v_in : (T)0;
  T *uo = io ? (T *)io->u_out : nullptr, *vo = io ? (T *)io->v_out : nullptr, *wo = io ? (T *)io->w_out : nullptr;
  if (io) {
    ProfScope ps(p, IBM_K_OUTFLOW, st, 2);
    const int ncol = p->nx * p->nz, nparts = ceil_div(ncol, kOutT);
    const size_t last = (size_t)(p->ny - 1) * ncol;
    const double step = ab * dt;
    double *part = (double *)p->work;
    IBM_CUDA_TRY(launch_pdl(k_outflow_update<T>, dim3(nparts), dim3(kOutT), 0, st, ncol, (const T *)(u + last),
                            (const T *)(v + last), (const T *)(w + last), uo, vo, wo, v,
                            (T)(step * io->c_out * 2.0 * g.ihy), (T)(step * io->c_out * g.ihy), v_lo, part));
    IBM_CUDA_TRY(launch_pdl(k_outflow_shift<T>, dim3(nparts), dim3(kOutT), 0, st, ncol, vo, io->v_in,
                            (const double *)part, nparts, 1.0 / ncol));
  }
  // E1
  {
    ProfScope ps(p, IBM_K_EXPLICIT, st);
    const dim3 eg(ceil_div(p->nx, kExTX), ceil_div(p->nz, kExTZ), ceil_div(p->ny, kExJC));
    if (io)
      IBM_CUDA_TRY(launch_pdl(k_explicit<T, true>, eg, dim3(kExTX, kExTZ), 0, st, g, u, v, w, pr, (T *)s->Nu,
                              (T *)s->Nv, (T *)s->Nw, du, dv, dw, (T)(ab * nu), (T)ab, (T)gm, (T)zt, (T)dt, v_lo,
                              (const T *)uo, (const T *)vo, (const T *)wo));
    else
      IBM_CUDA_TRY(launch_pdl(k_explicit<T, false>, eg, dim3(kExTX, kExTZ), 0, st, g, u, v, w, pr, (T *)s->Nu,
                              (T *)s->Nv, (T *)s->Nw, du, dv, dw, (T)(ab * nu), (T)ab, (T)gm, (T)zt, (T)dt, (T)0,
                              (const T *)nullptr, (const T *)nullptr, (const T *)nullptr));
  }
  // L2 + L1
  if (nmk > 0) {
    T *F = mk->F ? (T *)mk->F : (T *)p->mkbuf;
    {
      // L2 (rigid marker motion at the stage start time) fused with L1's
      // interpolation and force
      ProfScope ps(p, IBM_K_INTERP, st);
      IBM_CUDA_TRY(launch_interp<T>(p, nmk, (const T *)mk->X, u, v, w, du, dv, dw, nullptr, (const T *)mk->Ud,
                                    1.0 / dt, F, (const T *)mk->X0, (T *)mk->X, (T *)mk->Ud, mk->motion, mk->params,
                                    s->t, st));
    }
    {
      ProfScope ps(p, IBM_K_SPREAD, st);
      IBM_CUDA_TRY(launch_spread<T>(p, nmk, (const T *)mk->X, F, (const T *)mk->dV, du, dv, dw, dt, st));
    }
  }
  // S1: Helmholtz, increment form, u* written over u; the three components
  // go through the same launches
  {
    const int bcs[3] = {IBM_FIELD_CELL_DIRICHLET, IBM_FIELD_FACE_DIRICHLET, IBM_FIELD_CELL_DIRICHLET};
    const void *in3[3] = {du, dv, dw};
    void *out3[3] = {u, v, w};
    const void *add3[3] = {u, v, w};
    if ((rc = plan_solve_fields(p, cH, 3, bcs, in3, out3, add3, st))) return rc;
  }
  // E2
  const ff fx = ff_host(g.ihx), fy = ff_host(g.ihy), fz = ff_host(g.ihz);
  {
    ProfScope ps(p, IBM_K_DIVERGENCE, st);
    IBM_CUDA_TRY(launch_divergence<T>(g, L3, u, v, w, rhs, 1.0 / (ab * dt), fx, fy, fz, info ? p->dsc + 9 : nullptr,
                                      v_lo, (const T *)vo, st));
  }
  // S2
  if ((rc = plan_solve(p, 0, 0.0, 0, rhs, phi, nullptr, st, nullptr))) return rc;
  // E3
  {
    ProfScope ps(p, IBM_K_PROJECT, st);
    IBM_CUDA_TRY(launch_project<T>(g, L3, u, v, w, pr, phi, ab * dt, cH, v_lo, st));
  }
  if (info) {
    IBM_CUDA_TRY(cudaEventRecord(p->ev1, st));
    IBM_CUDA_TRY(launch_divergence<T>(g, L3, u, v, w, (T *)nullptr, 1.0, fx, fy, fz, p->dsc + 8, v_lo,
                                      (const T *)vo, st));
    IBM_CUDA_TRY(cudaMemcpyAsync(p->hsc, p->dsc, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
    IBM_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    IBM_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    trace.read(info->phase_ms);
    if ((rc = plan_status(p, st))) return rc;
    info->rel_residual = -1.0;
    info->removed_mean = p->hsc[0];
    info->div_max = p->hsc[8];
    info->div_before = p->hsc[9];
    info->t_ms = ms;
    info->refine_iters = p->precision == IBM_FP32_REFINED ? p->refine : 0;
  }
  s->t += ab * dt;
  return IBM_OK;
}

}  // namespace ibm

using namespace ibm;

static int substep_entry(ibm_plan plan, ibm_state *st, const ibm_inout *io, int rk_stage, double dt, double nu,
                         ibm_markers *mk, void *stream, ibm_info *info) {
  if (!plan || !st) return set_error(IBM_ERR_ARG, "ibm_substep: NULL plan or state");
  if (plan->bc != IBM_BC_PXZ_WALL_Y)
    return set_error(IBM_ERR_UNSUPPORTED, "ibm_substep: the RK stage is built for the wall-bounded branch only");
  if (rk_stage < 1 || rk_stage > 3) return set_error(IBM_ERR_ARG, "ibm_substep: rk_stage %d", rk_stage);
  if (!(dt > 0) || !std::isfinite(dt) || !(nu > 0) || !std::isfinite(nu))
    return set_error(IBM_ERR_ARG, "ibm_substep: dt and nu must be finite and > 0");
  void *fields[] = {st->u, st->v, st->w, st->p, st->Nu, st->Nv, st->Nw};
  for (void *f : fields)
    if (!f || !aligned_to(f, 16)) return set_error(IBM_ERR_ARG, "ibm_substep: NULL or non-16-byte-aligned field");
  if (mk && mk->n > 0) {
    if (!mk->X0 || !mk->dV || !mk->X || !mk->Ud)
      return set_error(IBM_ERR_ARG, "ibm_substep: markers need X0, dV, X and Ud");
    if (mk->motion < IBM_MOTION_STATIC || mk->motion > IBM_MOTION_HEAVE)
      return set_error(IBM_ERR_ARG, "ibm_substep: motion %d", mk->motion);
    if (mk->motion == IBM_MOTION_HEAVE && !(mk->params[1] > 0))
      return set_error(IBM_ERR_ARG, "ibm_substep: heave period must be > 0");
    if (mk->n > (1 << 26)) return set_error(IBM_ERR_ARG, "ibm_substep: too many markers");
  } else if (mk && mk->n < 0) {
    return set_error(IBM_ERR_ARG, "ibm_substep: negative marker count");
  }
  if (io) {
    if (!std::isfinite(io->v_in) || !std::isfinite(io->c_out) || io->c_out < 0)
      return set_error(IBM_ERR_ARG, "ibm_substep_inout: v_in must be finite and c_out finite and >= 0");
    const void *planes[] = {io->u_out, io->v_out, io->w_out};
    for (const void *f : planes)
      if (!f || !aligned_to(f, 16))
        return set_error(IBM_ERR_ARG, "ibm_substep_inout: NULL or non-16-byte-aligned outlet plane");
  }
  if (plan->precision == IBM_FP64)
    return substep_t<double>(plan, st, io, rk_stage, dt, nu, mk, (cudaStream_t)stream, info);
  return substep_t<float>(plan, st, io, rk_stage, dt, nu, mk, (cudaStream_t)stream, info);
}

namespace ibm {
double stage_time_advance(int rk_stage, double dt) { return (kAlpha[rk_stage - 1] + kBeta[rk_stage - 1]) * dt; }

int substep_checked(ibm_plan_s *p, ibm_state *st, int rk_stage, double dt, double nu, ibm_markers *mk,
                    cudaStream_t stream) {
  return substep_entry(p, st, nullptr, rk_stage, dt, nu, mk, stream, nullptr);
}

int prepare_substep(ibm_plan_s *p, int nmk) {
  int rc = ensure_substep_buffers(p, nmk);
  if (rc) return rc;
  for (int b = 0; b < 2; ++b) {  // the spectra of the stage's three-field Helmholtz launches
    if (!p->Sx[b]) {
      cudaError_t e = cudaMalloc(&p->Sx[b], p->nspec * 2 * p->esz);
      if (e != cudaSuccess) { p->Sx[b] = nullptr; return cuda_error(e, "field spectrum"); }
      p->bytes += p->nspec * 2 * p->esz;
    }
  }
  return IBM_OK;
}
}  // namespace ibm

extern "C" int ibm_substep(ibm_plan plan, ibm_state *st, int rk_stage, double dt, double nu, ibm_markers *mk,
                           void *stream, ibm_info *info) {
  return substep_entry(plan, st, nullptr, rk_stage, dt, nu, mk, stream, info);
}

extern "C" int ibm_substep_inout(ibm_plan plan, ibm_state *st, const ibm_inout *io, int rk_stage, double dt,
                                 double nu, ibm_markers *mk, void *stream, ibm_info *info) {
  if (!io) return set_error(IBM_ERR_ARG, "ibm_substep_inout: NULL inflow-outflow data");
  return substep_entry(plan, st, io, rk_stage, dt, nu, mk, stream, info);
}
